"""Pins for the oracle's Algorithm 3 (lagged-diffusivity fixed point around MLSQR)."""
import numpy as np
import pytest

import oracle as O


def _dense(apply, shape):
    n = int(np.prod(shape))
    return np.stack([np.asarray(apply(np.eye(n)[i].reshape(shape))).ravel() for i in range(n)], 1)


def _fd(n):
    return np.eye(n, k=1) - np.eye(n)


def test_tikhonov_full_solve_is_direct_normal_equation_solve():
    """r = t^2/2 gives kappa = 1 and the linear problem (1.7)-(1.8): with an exact M^{-1}
    and enough inner iterations every outer step returns (A^T A + tau D^T D)^{-1} A^T g."""
    shape = (8, 10)
    rng = np.random.default_rng(21)
    op = O.Operator("blur", shape, sigma=(1.0, 1.4), radius=(3, 4))
    g = op.A(rng.uniform(0, 1, shape)) + 0.01 * rng.standard_normal(shape)
    tau = 0.05
    out = O.solve(op, g, "tikhonov", 1.0, tau, n_outer=2, n_inner=200, levels=1)
    Dx = np.kron(np.eye(8), _fd(10))
    Dy = np.kron(_fd(8), np.eye(10))
    A = _dense(op.A, shape)
    fd = np.linalg.solve(A.T @ A + tau * (Dx.T @ Dx + Dy.T @ Dy), A.T @ g.ravel())
    assert np.linalg.norm(out["f"].ravel() - fd) <= 1e-9 * np.linalg.norm(fd)
    assert out["R_hist"][0] == 0.0
    assert out["R_hist"][-1] == pytest.approx(0.5 * ((Dx @ fd) ** 2 + (Dy @ fd) ** 2).sum(), rel=1e-8)
    assert out["resid_hist"][-1] == pytest.approx(np.linalg.norm(g.ravel() - A @ fd), rel=1e-8)


def test_outer_steps_restart_and_record():
    shape = (16, 16)
    rng = np.random.default_rng(22)
    op = O.Operator("blur", shape, sigma=(1.5, 1.5), radius=(4, 4))
    f0 = np.zeros(shape)
    f0[4:12, 3:9] = 1.0
    g = op.A(f0) + 0.01 * rng.standard_normal(shape)
    out = O.solve(op, g, "tv", 0.05, 0.0, n_outer=4, n_inner=6, levels=3)
    assert out["status"] == 0
    # f^0 = 0: R(0) = N T for smoothed TV
    assert out["R_hist"][0] == pytest.approx(256 * 0.05)
    # the inner solve restarts from f = 0 (Sec. 4.3): each step's first residual estimate
    # is below ||g|| and the run of one outer step reproduces the first row
    one = O.solve(op, g, "tv", 0.05, 0.0, n_outer=1, n_inner=6, levels=3)
    assert np.array_equal(one["rbar_hist"][0], out["rbar_hist"][0])
    for k in range(4):
        assert out["rbar_hist"][k][0] < np.linalg.norm(g)
        # tau = 0: ||rbar_i|| is the true residual, non-increasing within a step
        assert np.all(np.diff(out["rbar_hist"][k]) <= 1e-12)
    # tau = 0: the last estimate of each step equals ||g - A f^k||
    assert out["rbar_hist"][-1][-1] == pytest.approx(out["resid_hist"][-1], rel=1e-8)


def test_lagged_diffusivity_fixed_point():
    """With an exact M^{-1}, tau > 0 and converged inner solves, Algorithm 3 is lagged
    diffusivity (Sec. 4.1): f^k approaches a solution of (4.1), (A^T A + tau M_f) f = A^T g."""
    shape = (12, 12)
    rng = np.random.default_rng(23)
    op = O.Operator("blur", shape, sigma=(1.2, 1.2), radius=(3, 3))
    f0 = np.zeros(shape)
    f0[3:9, 4:10] = 1.0
    g = op.A(f0) + 0.01 * rng.standard_normal(shape)
    tau, T = 2e-3, 0.1
    A = _dense(op.A, shape)

    def grad_residual(f):
        kappa, _ = O.diffusivity(f, "tv", T, kfloor=1e-4)
        return np.linalg.norm(A.T @ (A @ f.ravel() - g.ravel()) + tau * O.apply_M(kappa, f).ravel())

    res = [grad_residual(O.solve(op, g, "tv", T, tau, n_outer=k, n_inner=300, levels=1)["f"])
           for k in (1, 4, 30)]
    scale = np.linalg.norm(A.T @ g.ravel())
    assert res[2] < res[1] < res[0]
    assert res[2] < 1e-6 * scale


@pytest.mark.parametrize("reg,tau", [("tv", 0.0), ("tv", 1e-3), ("pm_log", 0.0), ("pm_log", 1e-3)])
def test_regulariser_rises_then_saturates_and_the_level_drops(reg, tau):
    """The qualitative behaviour of Sec. 4.3 (Fig. 4.3): within an outer step R(f_i) rises with
    the inner iterations and levels off; over the first outer steps the level it reaches drops
    (not at every step: with tau > 0 the second TV level here lies 0.1% above the first, the
    fourth 1.8% below it).  A fixed point that never updates kappa would repeat the first level."""
    shape = (32, 32)
    rng = np.random.default_rng(31)
    f0 = np.zeros(shape)
    f0[6:20, 5:16] = 1.0
    f0[15:28, 12:27] = 0.5
    yy, xx = np.mgrid[:32, :32]
    f0[(yy - 9) ** 2 + (xx - 24) ** 2 < 25] = 0.8
    op = O.Operator("blur", shape, sigma=(1.5, 1.5), radius=(5, 5))
    Af = op.A(f0)
    g = Af + 0.01 * np.linalg.norm(Af) / np.sqrt(Af.size) * rng.standard_normal(shape)
    T, n = 0.05, 20
    # inner iterates of the first outer step: MLSQR restarts from 0, so the run of i iterations
    # ends at f_i
    mg = O.Multigrid(O.diffusivity(np.zeros(shape), reg, T)[0], 3, 2, 1)
    Rs = np.array([O.diffusivity(O.mlsqr(op, g, tau, i, prec=mg)[0], reg, T)[1] for i in range(1, n + 1)])
    inc = np.diff(Rs)
    assert Rs[-1] > Rs[0]
    assert inc[-5:].mean() < 0.25 * inc[:5].mean()
    out = O.solve(op, g, reg, T, tau, n_outer=4, n_inner=n, levels=3)
    assert out["R_hist"][1] == pytest.approx(Rs[-1], rel=1e-12)
    assert out["R_hist"][4] < 0.995 * out["R_hist"][1]


@pytest.mark.parametrize("reg,tau", [("tv", 1e-3), ("pm_log", 0.0), ("pm_exp", 2e-3)])
def test_whole_pipeline_against_dense_restatement(reg, tau):
    """Algorithm 3 with the V-cycle priorconditioner against a dense restatement written here:
    explicit A and forward differences, kappa = r'(t)/t from its closed form (1.4)/(1.5) with the
    floor, P as a dense matrix from the oracle's V-cycle (pinned on its own), and each inner solve
    as scipy's LSQR on A L^{-1} with L^T L = P^{-1} (Algorithm 1), restarted from 0 every outer
    step (Sec. 4.3).  Checks the glue: kappa from f^{k-1}, the restart, R(f^k) and ||g - A f^k||."""
    from scipy.sparse.linalg import lsqr

    shape, T, levels, nu, cycles, n_outer, n_inner, kfloor = (8, 8), 0.1, 2, 2, 1, 3, 6, 1e-4
    rng = np.random.default_rng(24)
    op = O.Operator("blur", shape, sigma=(1.0, 1.2), radius=(2, 3))
    f0 = np.zeros(shape)
    f0[2:6, 1:5] = 1.0
    f0[4:8, 5:8] = 0.5
    g = op.A(f0) + 0.01 * rng.standard_normal(shape)
    A = _dense(op.A, shape)
    Dx = np.kron(np.eye(8), _fd(8))
    Dy = np.kron(_fd(8), np.eye(8))

    def kappa_R(f):
        t = np.sqrt((Dx @ f) ** 2 + (Dy @ f) ** 2)
        if reg == "tv":
            k, r, k0 = 1.0 / np.sqrt(T * T + t * t), np.sqrt(T * T + t * t), 1.0 / T
        elif reg == "pm_log":
            k, r, k0 = 1.0 / (1.0 + (t / T) ** 2), 0.5 * T * T * np.log1p((t / T) ** 2), 1.0
        else:
            k, r, k0 = np.exp(-(t / T) ** 2), 0.5 * T * T * (1.0 - np.exp(-(t / T) ** 2)), 1.0
        return np.maximum(k, kfloor * k0), r.sum()

    f = np.zeros(64)
    R_hist, resid, last_rbar = [kappa_R(f)[1]], [], []
    for _ in range(n_outer):
        kappa = kappa_R(f)[0]
        P = _dense(O.Multigrid(kappa.reshape(shape), levels, nu, cycles).apply, shape)
        L = np.linalg.cholesky(np.linalg.inv(0.5 * (P + P.T))).T
        r = lsqr(A @ np.linalg.inv(L), g.ravel(), damp=np.sqrt(tau), iter_lim=n_inner, atol=0, btol=0, conlim=0)
        f = np.linalg.solve(L, r[0])
        R_hist.append(kappa_R(f)[1])
        resid.append(np.linalg.norm(g.ravel() - A @ f))
        last_rbar.append(r[4])
    out = O.solve(op, g, reg, T, tau, n_outer, n_inner, levels, nu, cycles, kfloor=kfloor)
    assert out["status"] == 0
    assert np.linalg.norm(out["f"].ravel() - f) <= 1e-9 * np.linalg.norm(f)
    assert np.allclose(out["R_hist"], R_hist, rtol=1e-10, atol=0)
    assert np.allclose(out["resid_hist"], resid, rtol=1e-9, atol=0)
    assert np.allclose(out["rbar_hist"][:, -1], last_rbar, rtol=1e-9, atol=0)
