"""Guard bands around the workspace: no kernel writes past either end of a workspace allocation.

With PLSQR_GUARD=1 at plsqr_create every allocation of the handle carries 256 bytes of a fixed
pattern on each side; plsqr_check_guards reads them back.  Each case runs the batched solve, the
single-operator entry points (forward and adjoint maps, diffusivity, priorconditioner, M_f,
MLSQR) and, for the single-precision 2D blur, the slots of continuous batching on a second
handle, then checks every band.  The banded handles must also give bit for bit the results of
handles without bands (the regions move, the arithmetic does not).  Collected last: a failure
here stops no other test.
"""
import numpy as np
import pytest

import oracle as O
from paper_1308_6634_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1308_6634_gb300 import build
    build.build()


CASES = {
    "blur2d_fp32": synth.Workload("blur2d_fp32", "blur", (128, 128), "fp32", "pm_log", 5e-2, 1e-3, 3, 8, levels=4,
                                  nu=2, cycles=1, sigma=(4.0, 4.0), radius=(12, 12),
                                  phantom=dict(type="rects_disks", rects=10, disks=6)),
    "blur2d_fp64": synth.Workload("blur2d_fp64", "blur", (64, 64), "fp64", "tv", 1e-2, 5e-3, 3, 8, levels=3, nu=2,
                                  cycles=2, sigma=(2.0, 2.0), radius=(6, 6),
                                  phantom=dict(type="rects_disks", rects=6, disks=4)),
    "inpaint3d_fp32": synth.Workload("inpaint3d_fp32", "blur_mask", (32, 32, 32), "fp32", "tv", 1e-2, 0.0, 2, 6,
                                     levels=3, nu=2, cycles=1, sigma=(3.0, 3.0, 5.0), radius=(9, 9, 15),
                                     noise=0.005, missing=0.15, phantom=dict(type="ellipsoids", count=6)),
    "tomo_fp32": synth.Workload("tomo_fp32", "joseph", (64, 64), "fp32", "pm_exp", 2e-2, 0.0, 2, 6, levels=3, nu=2,
                                cycles=1, n_angles=60, n_bins=93, phantom=dict(type="ellipses", count=5)),
}


def dev(x, prec):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=torch.float64 if prec == "fp64" else torch.float32).cuda()


def _problem(W, seed):
    f, mask, z = W.inputs(seed)
    op = O.Operator(W.kind, W.shape, sigma=W.sigma, radius=W.radius, mask=mask, n_angles=W.n_angles,
                    n_bins=W.n_bins)
    return f, op, synth.add_noise(op.A(f), W.noise, z), mask


def _solver(W, mask, guard, monkeypatch):
    from paper_1308_6634_gb300 import plsqr
    if guard:
        monkeypatch.setenv("PLSQR_GUARD", "1")
    S = plsqr.Solver(W.shape, W.precision, levels=W.levels, sweeps=W.nu, cycles=W.cycles, max_batch=2)
    monkeypatch.delenv("PLSQR_GUARD", raising=False)
    S.set_operator(W.kind, sigma=W.sigma, radius=W.radius, mask=mask, n_angles=W.n_angles, n_bins=W.n_bins)
    return S


def _run(W, guard, monkeypatch):
    """Everything a handle can do on this workload; returns (handles, list of result arrays)."""
    monkeypatch.delenv("PLSQR_GUARD", raising=False)
    (f0, op, g0, mask), (_, _, g1, _) = _problem(W, 0), _problem(W, 1)
    S = _solver(W, mask, guard, monkeypatch)
    handles = [S]
    p = W.precision
    out = []
    fs, infos = S.solve_batch([dev(g0, p), dev(g1, p)], [W.reg] * 2, [W.T] * 2, [W.tau] * 2, W.n_outer, W.n_inner)
    out += [t.double().cpu().numpy() for t in fs] + [i["rbar_hist"] for i in infos]
    out.append(S.apply_A(dev(f0, p)).double().cpu().numpy())
    out.append(S.apply_At(dev(g0, p)).double().cpu().numpy())
    kappa, _ = S.diffusivity(dev(f0 + 0.01 * np.random.default_rng(2).standard_normal(W.shape), p), W.reg, W.T)
    S.prec_setup(kappa)
    b = dev(np.random.default_rng(3).standard_normal(W.shape), p)
    out.append(S.prec_apply(b).double().cpu().numpy())
    out.append(S.apply_M(b).double().cpu().numpy())
    f, hist, _ = S.mlsqr(dev(g0, p), W.tau, 4)
    out += [f.double().cpu().numpy(), hist]
    if W.kind == "blur" and len(W.shape) == 2 and p == "fp32":  # slots of continuous batching
        S2 = _solver(W, mask, guard, monkeypatch)
        handles.append(S2)
        S2.slot_start(1, dev(g1, p), W.reg, W.T, W.tau, 2, W.n_inner)
        for _ in range(2):
            S2.step()
        fsl, info = S2.slot_finish(1, 2, W.n_inner)
        out += [fsl.double().cpu().numpy(), info["rbar_hist"]]
    torch.cuda.synchronize()
    return handles, out


@pytest.mark.parametrize("case", sorted(CASES))
def test_guard_bands_stay_intact(case, monkeypatch):
    W = CASES[case]
    handles, got = _run(W, True, monkeypatch)
    for S in handles:
        checked, bad = S.check_guards()
        assert checked >= 10 and bad == 0, (checked, bad)
    plain, ref = _run(W, False, monkeypatch)
    assert all(S.check_guards() == (0, 0) for S in plain)
    assert len(got) == len(ref)
    for k, (a, b) in enumerate(zip(got, ref)):
        assert np.array_equal(a, b, equal_nan=True), k
