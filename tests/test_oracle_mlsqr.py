"""Pins for the oracle's MLSQR (Algorithm 2) against independent routines.

Sec. 3.2: MLSQR with P = M^{-1} (here any fixed SPD P, M := P^{-1}) produces the iterates
of plain LSQR on the transformed problem A L^{-1} with L^T L = M, mapped back by L^{-1}
(Algorithm 1), and of CG on the normal equations (3.2) in the M inner product.  scipy's
LSQR (Paige-Saunders, with its own damping rotation) and CG serve as the independent
implementations.
"""
import numpy as np
import pytest
from scipy.sparse.linalg import LinearOperator, cg, lsqr

import oracle as O


def _problem(shape=(12, 12), seed=11):
    rng = np.random.default_rng(seed)
    op = O.Operator("blur", shape, sigma=(0.7, 0.9), radius=(2, 2))
    f = np.zeros(shape)
    f[3:8, 2:9] = 1.0
    f[7:11, 6:11] = 0.4
    g = op.A(f) + 0.01 * rng.standard_normal(shape)
    kappa, _ = O.diffusivity(f, "pm_log", 0.3)
    return op, g, kappa


def _dense(apply, shape):
    n = int(np.prod(shape))
    return np.stack([np.asarray(apply(np.eye(n)[i].reshape(shape))).ravel() for i in range(n)], 1)


@pytest.mark.parametrize("levels,tau", [(1, 0.0), (1, 0.05), (2, 0.0), (3, 0.02)])
def test_mlsqr_equals_lsqr_on_transformed_problem(levels, tau):
    op, g, kappa = _problem()
    shape = op.shape
    mg = O.Multigrid(kappa, levels=levels, nu=2, cycles=1)
    P = _dense(mg.apply, shape)
    A = _dense(op.A, shape)
    Minv = 0.5 * (P + P.T)
    L = np.linalg.cholesky(np.linalg.inv(Minv)).T  # L^T L = P^{-1}
    Ahat = A @ np.linalg.inv(L)
    # short runs: with loss of orthogonality the iterates of two correct LSQR codes drift
    # apart by rounding; long runs are pinned by convergence to the direct solve below
    for k in [1, 2, 4, 6]:
        f, hist, st = O.mlsqr(op, g, tau, k, prec=mg)
        assert st == 0 and len(hist) == k
        r = lsqr(Ahat, g.ravel(), damp=np.sqrt(tau), iter_lim=k, atol=0, btol=0, conlim=0)
        fref = np.linalg.solve(L, r[0])
        assert np.linalg.norm(f.ravel() - fref) <= 1e-9 * np.linalg.norm(fref), k
        # ||rbar_k|| of the damped problem: scipy's r2norm
        assert hist[-1] == pytest.approx(r[4], rel=1e-10)


@pytest.mark.parametrize("tau", [0.0, 0.1])
def test_identity_preconditioner_is_plain_lsqr(tau):
    op, g, _ = _problem()
    A = _dense(op.A, op.shape)
    for k in [1, 3, 6]:
        f, hist, _ = O.mlsqr(op, g, tau, k, prec=None)
        r = lsqr(A, g.ravel(), damp=np.sqrt(tau), iter_lim=k, atol=0, btol=0, conlim=0)
        assert np.linalg.norm(f.ravel() - r[0]) <= 1e-10 * np.linalg.norm(r[0])
        assert hist[-1] == pytest.approx(r[4], rel=1e-10)


def test_mlsqr_equals_pcg_on_normal_equations():
    """PCG on (A^T A + tau P^{-1}) f = A^T g with preconditioner P (Sec. 3, eq. 3.2)."""
    op, g, kappa = _problem()
    shape, n = op.shape, int(np.prod(op.shape))
    tau = 0.03
    mg = O.Multigrid(kappa, levels=2)
    P = _dense(mg.apply, shape)
    A = _dense(op.A, shape)
    K = A.T @ A + tau * np.linalg.inv(0.5 * (P + P.T))
    b = A.T @ g.ravel()
    iterates = []
    cg(K, b, x0=np.zeros(n), rtol=1e-30, atol=0, maxiter=6,
       M=LinearOperator((n, n), matvec=lambda x: P @ x), callback=lambda xk: iterates.append(xk.copy()))
    for k, xk in enumerate(iterates, start=1):
        f, _, _ = O.mlsqr(op, g, tau, k, prec=mg)
        assert np.linalg.norm(f.ravel() - xk) <= 1e-8 * np.linalg.norm(xk), k


def test_residual_estimate_monotone_and_converges_to_direct_solve():
    op, g, kappa = _problem(shape=(8, 8))
    tau = 0.02
    mg = O.Multigrid(kappa, levels=1)  # exact M^{-1}
    f, hist, st = O.mlsqr(op, g, tau, 200, prec=mg)
    assert st in (0, 4)
    assert np.all(np.diff(hist) <= 1e-12 * hist[0])
    A = _dense(op.A, op.shape)
    M = _dense(lambda x: O.apply_M(kappa, x), op.shape)
    fd = np.linalg.solve(A.T @ A + tau * M, A.T @ g.ravel())
    assert np.linalg.norm(f.ravel() - fd) <= 1e-9 * np.linalg.norm(fd)


def test_denoising_special_case():
    """A = I: the converged solve is (I + tau M) f = g."""
    rng = np.random.default_rng(12)
    shape = (6, 8)
    op = O.Operator("identity", shape)
    g = rng.uniform(0, 1, shape)
    kappa = rng.uniform(0.2, 1.0, shape)
    mg = O.Multigrid(kappa, levels=1)
    f, _, _ = O.mlsqr(op, g, 0.5, 120, prec=mg)
    M = _dense(lambda x: O.apply_M(kappa, x), shape)
    fd = np.linalg.solve(np.eye(48) + 0.5 * M, g.ravel())
    assert np.linalg.norm(f.ravel() - fd) <= 1e-10 * np.linalg.norm(fd)


def test_zero_data_breakdown():
    op, _, kappa = _problem()
    f, hist, st = O.mlsqr(op, np.zeros(op.shape), 0.0, 5, prec=O.Multigrid(kappa, 2))
    assert st == 4 and len(hist) == 0 and np.all(f == 0)


def test_priorconditioning_reaches_discrepancy_sooner():
    """Sec. 3.5 (1D deconvolution, ideal Perona-Malik prior): S4 is met in fewer MLSQR
    iterations with the priorconditioner than without (the paper reports 9 vs 16)."""
    n = 512
    x = (np.arange(n) + 0.5) / n
    f = np.where((x > 0.15) & (x < 0.35), 1.0, 0.0) + np.where((x > 0.55) & (x < 0.8), 0.5, 0.0)
    f += np.where((x > 0.65) & (x < 0.7), 0.4, 0.0)
    sig = 0.03 * n  # sigma_f = 0.03 on [0, 1]
    op = O.Operator("blur", (n,), sigma=(sig,), radius=(int(np.ceil(4 * sig)),))
    rng = np.random.default_rng(13)
    noise = 0.01 * rng.standard_normal(n)
    g = op.A(f) + noise
    delta, eta = np.linalg.norm(noise), 1.1
    kappa, _ = O.diffusivity(f, "pm_log", 0.005)
    mg = O.Multigrid(kappa, levels=1)

    def first_below(prec):
        for k in range(1, 80):
            fk, _, _ = O.mlsqr(op, g, 0.0, k, prec=prec)
            if np.linalg.norm(g - op.A(fk)) <= eta * delta:
                return k
        return 10 ** 6

    kp, ku = first_below(mg), first_below(None)
    assert kp < ku


@pytest.mark.parametrize("levels", [1, 3])
def test_iterates_of_every_tau_lie_in_one_krylov_space(levels):
    """Sec. 2.1 / 3.3: K_k(P A^T A, P A^T g) does not depend on tau (shift invariance), so the k-th
    MLSQR iterate of every damping parameter lies in that one space.  The space is built here by
    dense products, independently of the oracle's bidiagonalisation; projecting each iterate on it
    leaves rounding only, while the iterates themselves differ between the values of tau."""
    op, g, kappa = _problem()
    shape = op.shape
    mg = O.Multigrid(kappa, levels=levels, nu=2, cycles=1)
    P = _dense(mg.apply, shape)
    A = _dense(op.A, shape)
    k = 4
    K = [P @ (A.T @ g.ravel())]
    for _ in range(k - 1):
        K.append(P @ (A.T @ (A @ K[-1])))
    Q, _ = np.linalg.qr(np.stack(K, 1))
    fs = []
    for tau in (0.0, 1e-3, 0.05, 1.0):
        f, _, st = O.mlsqr(op, g, tau, k, prec=mg)
        assert st == 0
        v = f.ravel()
        assert np.linalg.norm(v - Q @ (Q.T @ v)) <= 1e-8 * np.linalg.norm(v), tau
        fs.append(v)
    assert np.linalg.norm(fs[-1] - fs[0]) > 1e-2 * np.linalg.norm(fs[0])  # the damping does change the iterate


def _cg_damped_normal_equations(A, g, tau, k):
    """k steps of textbook CG (Hestenes-Stiefel) on (A^T A + tau I) f = A^T g from f = 0."""
    b = A.T @ g
    x = np.zeros_like(b)
    r = b.copy()
    p = r.copy()
    rr = float(r @ r)
    for _ in range(k):
        q = A.T @ (A @ p) + tau * p
        a = rr / float(p @ q)
        x = x + a * p
        r = r - a * q
        rr_new = float(r @ r)
        p = r + (rr_new / rr) * p
        rr = rr_new
    return x


@pytest.mark.parametrize("tau", [0.0, 0.05])
def test_plain_lsqr_equals_cg_on_the_normal_equations(tau):
    """Sec. 3: LSQR is CG on the (damped) normal equations, carried out on the bidiagonal form;
    with P = I the iterates of MLSQR are those of CG on (A^T A + tau I) f = A^T g."""
    op, g, _ = _problem()
    A = _dense(op.A, op.shape)
    for k in [1, 2, 3, 5, 7]:
        f, _, st = O.mlsqr(op, g, tau, k, prec=None)
        ref = _cg_damped_normal_equations(A, g.ravel(), tau, k)
        assert st == 0
        assert np.linalg.norm(f.ravel() - ref) <= 1e-9 * np.linalg.norm(ref), k
