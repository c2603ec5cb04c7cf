"""The oracle's stopping rules (Sec. 3.4 S4, Sec. 4.1 / Algorithm 3 step 5) against properties that
the paper fixes, checked with the forward map applied independently of the solver."""
import numpy as np
import pytest

import oracle as O
from paper_1308_6634_gb300 import synth


def _problem(n=48, sigma=2.0, R=6, noise=0.01, seed=0):
    f = synth.phantom_rects_disks(n, 6, 4, seed)
    op = O.Operator("blur", (n, n), sigma=(sigma, sigma), radius=(R, R))
    Af = op.A(f)
    z = synth.standard_noise((n, n), seed + 1)
    e = noise * np.linalg.norm(Af) / np.sqrt(Af.size) * z
    return op, Af + e, np.linalg.norm(e)


def _resid(op, g, f):
    return np.linalg.norm(g - op.A(f))


@pytest.mark.parametrize("eta", [1.1, 1.5, 3.0])
def test_s4_stops_at_the_first_iterate_inside_the_discrepancy_ball(eta):
    """tau = 0: the stopped iterate f_i has ||g - A f_i|| <= eta delta, and f_{i-1} (the same
    iteration run one step less) does not."""
    op, g, delta = _problem()
    kappa = O.diffusivity(np.zeros(op.shape), "tv", 1e-2)[0]
    mg = O.Multigrid(kappa, 3, 2, 1)
    f, hist, st = O.mlsqr_s4(op, g, 0.0, 200, eta * delta, prec=mg)
    i = len(hist)
    assert st == 0 and 1 < i < 200
    assert _resid(op, g, f) <= eta * delta * (1 + 1e-9)
    f_prev, _, _ = O.mlsqr(op, g, 0.0, i - 1, prec=mg)
    assert _resid(op, g, f_prev) > eta * delta
    # the estimate the rule uses is the true residual at tau = 0
    assert hist[-1] == pytest.approx(_resid(op, g, f), rel=1e-8)


def test_s4_with_damping_is_conservative():
    """tau > 0: the estimate ||rbar_i|| includes the penalty term, so the stopped iterate is
    inside the discrepancy ball as well."""
    op, g, delta = _problem()
    kappa = O.diffusivity(np.zeros(op.shape), "tv", 1e-2)[0]
    mg = O.Multigrid(kappa, 3, 2, 1)
    f, hist, st = O.mlsqr_s4(op, g, 1e-6, 300, 1.5 * delta, prec=mg)
    assert st == 0 and len(hist) < 300
    assert _resid(op, g, f) <= 1.5 * delta
    assert hist[-1] >= _resid(op, g, f) * (1 - 1e-9)


def test_s4_disabled_is_plain_mlsqr():
    op, g, _ = _problem()
    kappa = O.diffusivity(np.zeros(op.shape), "tv", 1e-2)[0]
    mg = O.Multigrid(kappa, 3, 2, 1)
    f1, h1, _ = O.mlsqr_s4(op, g, 1e-3, 12, 0.0, prec=mg)
    f2, h2, _ = O.mlsqr(op, g, 1e-3, 12, prec=mg)
    assert np.array_equal(f1, f2) and np.array_equal(h1, h2)


def test_outer_stop_on_the_relative_decrease_of_R():
    """The fixed point stops at the first f^j (j >= 2) whose R did not drop by more than r_rel;
    every earlier step dropped by more; the result is the plain solve run for j steps."""
    op, g, delta = _problem(n=32)
    r_rel = 0.15
    out = O.solve_stop(op, g, "pm_log", 5e-2, 1e-3, 12, 25, 3, 0.0, r_rel)
    j = out["outer_done"]
    R = out["R_hist"]
    assert out["status"] == 0 and 2 <= j < 12
    assert (R[j] - R[j - 1]) / R[j - 1] > -r_rel
    for l in range(2, j):
        assert (R[l] - R[l - 1]) / R[l - 1] <= -r_rel
    plain = O.solve(op, g, "pm_log", 5e-2, 1e-3, j, 25, 3)
    assert np.array_equal(plain["f"], out["f"])
    assert np.array_equal(plain["R_hist"][: j + 1], R[: j + 1])


def test_both_rules_together():
    op, g, delta = _problem(n=32)
    out = O.solve_stop(op, g, "tv", 1e-2, 0.0, 10, 60, 3, 1.1 * delta, 0.15)
    j = out["outer_done"]
    assert out["status"] == 0 and j >= 1
    for k in range(j):  # every inner solve stopped by S4 or by the cap
        h = out["rbar_hist"][k]
        n_run = int(np.sum(np.isfinite(h)))
        assert n_run == 60 or h[n_run - 1] <= 1.1 * delta
        assert n_run == 60 or np.all(h[: n_run - 1] > 1.1 * delta)
