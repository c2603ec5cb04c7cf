"""Pins for the oracle's V-cycle P, the fixed symmetric approximation of M^{-1} (Sec. 4.2).

A symmetric smoother mirrored between pre- and post-smoothing, R = P^T and an exact
coarse solve make P a fixed SPD operator, which priorconditioning needs (Sec. 4.2).
"""
import numpy as np
import pytest

import oracle as O


def _kappa(shape, seed=7, contrast=100.0):
    rng = np.random.default_rng(seed)
    f = np.zeros(shape)
    sl = tuple(slice(s // 4, 3 * s // 4) for s in shape)
    f[sl] = 1.0
    k = np.where(f > 0, 1.0, 1.0 / contrast) * rng.uniform(0.5, 1.5, size=shape)
    return k


@pytest.mark.parametrize("shape", [(8, 8), (4, 6, 8)])
def test_one_level_is_exact_inverse(shape, dense):
    kappa = _kappa(shape)
    mg = O.Multigrid(kappa, levels=1)
    P = dense(mg.apply, shape)
    M = dense(lambda x: O.apply_M(kappa, x), shape)
    assert np.abs(P @ M - np.eye(P.shape[0])).max() < 1e-11


@pytest.mark.parametrize("shape,levels,nu,cycles", [((16, 16), 3, 2, 1), ((16, 8), 4, 1, 2),
                                                    ((8, 8, 8), 3, 2, 1), ((8, 4, 8), 2, 1, 1)])
def test_vcycle_symmetric_positive_definite(shape, levels, nu, cycles, dense):
    kappa = _kappa(shape)
    mg = O.Multigrid(kappa, levels=levels, nu=nu, cycles=cycles)
    P = dense(mg.apply, shape)
    assert np.abs(P - P.T).max() < 1e-13 * np.abs(P).max()
    np.linalg.cholesky(0.5 * (P + P.T))
    # energy-norm contraction ||I - P M||_M < 1 (a convergent fixed linear iteration)
    M = dense(lambda x: O.apply_M(kappa, x), shape)
    Lm = np.linalg.cholesky(M)
    E = Lm.T @ (np.eye(M.shape[0]) - P @ M) @ np.linalg.inv(Lm.T)
    assert np.linalg.norm(E, 2) < 1.0


def test_cycles_compose(dense):
    shape = (16, 16)
    kappa = _kappa(shape)
    M = dense(lambda x: O.apply_M(kappa, x), shape)
    I = np.eye(M.shape[0])
    P1 = dense(O.Multigrid(kappa, 3, 2, 1).apply, shape)
    P3 = dense(O.Multigrid(kappa, 3, 2, 3).apply, shape)
    # x <- x + V(b - Mx) three times from 0: I - P3 M = (I - P1 M)^3
    assert np.abs((I - P3 @ M) - np.linalg.matrix_power(I - P1 @ M, 3)).max() < 1e-10
    # many cycles converge to M^{-1}
    P40 = dense(O.Multigrid(kappa, 3, 2, 40).apply, shape)
    assert np.abs(P40 @ M - I).max() < 1e-6


@pytest.mark.parametrize("shape", [(8, 12), (4, 6, 8)])
def test_galerkin_coarse_operator(shape, dense):
    """Coarse level operator = P^T M P with piecewise-constant prolongation P."""
    kappa = _kappa(shape)
    mg = O.Multigrid(kappa, levels=2)
    cshape = tuple(s // 2 for s in shape)
    nf, nc = int(np.prod(shape)), int(np.prod(cshape))
    Pm = np.zeros((nf, nc))
    for fi in range(nf):
        c = np.unravel_index(fi, shape)
        Pm[fi, np.ravel_multi_index(tuple(ci // 2 for ci in c), cshape)] = 1.0
    M = dense(lambda x: O.apply_M(kappa, x), shape)
    Mc = dense(lambda x: mg.level_apply(1, x), cshape)
    assert np.abs(Mc - Pm.T @ M @ Pm).max() < 1e-12


def test_invalid_sizes_rejected():
    with pytest.raises(ValueError):
        O.Multigrid(np.ones((12, 12)), levels=4)  # 12 not divisible by 8


def test_constant_kappa_poisson_two_grid_improves_smoother(dense):
    """With kappa = 1 the V-cycle beats the smoother alone in the energy norm."""
    shape = (32, 32)
    kappa = np.ones(shape)
    M = dense(lambda x: O.apply_M(kappa, x), shape)
    Lm = np.linalg.cholesky(M)
    I = np.eye(M.shape[0])

    def rate(P):
        return np.linalg.norm(Lm.T @ (I - P @ M) @ np.linalg.inv(Lm.T), 2)

    r1 = rate(dense(O.Multigrid(kappa, 1, 2, 1).apply, shape))
    r2 = rate(dense(O.Multigrid(kappa, 2, 2, 1).apply, shape))
    r5 = rate(dense(O.Multigrid(kappa, 5, 2, 1).apply, shape))
    assert r1 < 1e-10  # exact solve
    # piecewise-constant two-grid with Galerkin coarse operator: about 1/2 on Poisson
    assert r2 < 0.55
    # deeper hierarchies of this kind degrade but stay a contraction
    assert r2 < r5 < 0.9
