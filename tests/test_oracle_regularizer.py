"""Pins for the oracle's regulariser, diffusivity and weighted diffusion operator M_f.

Paper: r(t) of (1.3)-(1.5); kappa = r'(t)/t, the diffusivity of (1.13); M_f the
discrete form of -div(kappa grad) (Sec. 1.4), here sum_d D_d^T diag(kappa) D_d on the
tensor grid with forward differences and a ghost 0 beyond the high end of each axis.
"""
import numpy as np
import pytest

import oracle as O

REGS = ["tikhonov", "tv", "pm_log", "pm_exp"]


def test_special_values():
    T = 0.37
    # (1.3): kappa = 1 for every t; r(2) = 2
    assert O.kappa_of("tikhonov", T, 5.0) == 1.0
    assert O.r_of("tikhonov", T, 2.0) == pytest.approx(2.0, rel=1e-15)
    # (1.4) smoothed TV: r(0) = T, kappa(0) = 1/T, r(t) -> t for t >> T
    assert O.r_of("tv", T, 0.0) == pytest.approx(T, rel=1e-15)
    assert O.kappa_of("tv", T, 0.0) == pytest.approx(1.0 / T, rel=1e-15)
    assert O.r_of("tv", 1e-6, 3.0) == pytest.approx(3.0, rel=1e-10)
    # (1.5) left: r(T) = T^2 log(2)/2, kappa(T) = 1/2
    assert O.r_of("pm_log", T, T) == pytest.approx(0.5 * T * T * np.log(2.0), rel=1e-14)
    assert O.kappa_of("pm_log", T, T) == pytest.approx(0.5, rel=1e-15)
    # (1.5) right: r -> T^2/2 as t -> inf, kappa(T) = 1/e
    assert O.r_of("pm_exp", T, 50 * T) == pytest.approx(0.5 * T * T, rel=1e-14)
    assert O.kappa_of("pm_exp", T, T) == pytest.approx(np.exp(-1.0), rel=1e-15)
    # all r(0) = 0 except TV
    for reg in ["tikhonov", "pm_log", "pm_exp"]:
        assert O.r_of(reg, T, 0.0) == 0.0


@pytest.mark.parametrize("reg", REGS)
def test_kappa_is_rprime_over_t(reg):
    """kappa(t) * t must be the derivative of r (central differences of the oracle's r)."""
    T = 0.05
    for t in [1e-3, 0.01, 0.05, 0.2, 0.7]:
        h = 1e-6 * max(t, T)
        d = (O.r_of(reg, T, t + h) - O.r_of(reg, T, t - h)) / (2 * h)
        assert O.kappa_of(reg, T, t) * t == pytest.approx(d, rel=1e-7, abs=1e-12)


def _D(n):
    """1D forward difference with ghost 0 beyond the end: (D f)_i = f_{i+1} - f_i."""
    return np.eye(n, k=1) - np.eye(n)


def _Dd(shape, axis_from_x):
    """Forward difference along an axis (0 = x, fastest) of a C-order array of `shape`."""
    dims = list(shape)  # (.., ny, nx)
    mats = []
    for k, n in enumerate(dims):
        ax = len(dims) - 1 - k  # axis index counted from x
        mats.append(_D(n) if ax == axis_from_x else np.eye(n))
    out = mats[0]
    for m in mats[1:]:
        out = np.kron(out, m)
    return out


@pytest.mark.parametrize("shape", [(7,), (5, 6), (3, 4, 5)])
def test_M_equals_dense_DtKD(shape, dense):
    rng = np.random.default_rng(1)
    kappa = rng.uniform(0.1, 2.0, size=shape)
    M = dense(lambda x: O.apply_M(kappa, x), shape)
    ref = sum(_Dd(shape, d).T @ np.diag(kappa.ravel()) @ _Dd(shape, d) for d in range(len(shape)))
    assert np.abs(M - ref).max() < 1e-13
    assert np.linalg.eigvalsh(M).min() > 0  # SPD for kappa > 0


@pytest.mark.parametrize("shape", [(6, 7), (3, 4, 5)])
@pytest.mark.parametrize("reg", REGS)
def test_gradient_of_R_is_M_f_f(shape, reg):
    """The discrete Frechet derivative (1.12): grad R(f) = M_f f with kappa taken from f."""
    rng = np.random.default_rng(2)
    f = rng.uniform(0, 1, size=shape)
    h = rng.standard_normal(shape)
    T = 0.3
    kappa, _ = O.diffusivity(f, reg, T, kfloor=0.0)
    g_lin = float((h * O.apply_M(kappa, f)).sum())
    eps = 1e-6
    Rp = O.diffusivity(f + eps * h, reg, T, kfloor=0.0)[1]
    Rm = O.diffusivity(f - eps * h, reg, T, kfloor=0.0)[1]
    assert (Rp - Rm) / (2 * eps) == pytest.approx(g_lin, rel=1e-7)


def test_diffusivity_ghost_and_floor():
    # one cell: t = |0 - f0| (ghost value 0)
    for reg in REGS:
        k, R = O.diffusivity(np.array([0.3]), reg, 0.1, kfloor=0.0)
        assert k[0] == O.kappa_of(reg, 0.1, 0.3)
        assert R == O.r_of(reg, 0.1, 0.3)
    # PM-exp with a jump >> T underflows; the floor keeps kappa >= kfloor * kappa(0)
    f = np.zeros((4, 4))
    f[:, 2:] = 1.0
    k, _ = O.diffusivity(f, "pm_exp", 0.02, kfloor=1e-4)
    assert k.min() == pytest.approx(1e-4)
    assert k.max() == 1.0
    # TV, f = 0 everywhere: kappa = 1/T and R = N T
    k, R = O.diffusivity(np.zeros((5, 6)), "tv", 0.01)
    assert np.all(k == 100.0) and R == pytest.approx(30 * 0.01)


def _laplacian_stencil(x):
    """sum over axes of D^T D x written cell by cell: for each axis, (x - x_low) where a lower
    neighbour exists, plus (x - x_high) with x_high = 0 beyond the high end."""
    out = np.zeros_like(x)
    for idx in np.ndindex(*x.shape):
        v = 0.0
        for ax in range(x.ndim):
            lo, hi = list(idx), list(idx)
            lo[ax] -= 1
            hi[ax] += 1
            if lo[ax] >= 0:
                v += x[idx] - x[tuple(lo)]
            v += x[idx] - (x[tuple(hi)] if hi[ax] < x.shape[ax] else 0.0)
        out[idx] = v
    return out


@pytest.mark.parametrize("shape", [(5, 7), (3, 4, 5)])
@pytest.mark.parametrize("reg", REGS)
def test_first_priorconditioner_is_the_laplacian(shape, reg):
    """Sec. 4.3: Algorithm 3 starts from f = 0, where every gradient vanishes, so kappa is the
    constant kappa(0) (1, or 1/T for smoothed TV) and the first M_f is kappa(0) times the
    discrete Laplacian; R(0) = N r(0)."""
    T = 0.2
    kappa, R = O.diffusivity(np.zeros(shape), reg, T)
    k0 = 1.0 / T if reg == "tv" else 1.0
    assert np.all(kappa == k0)
    assert R == pytest.approx(np.prod(shape) * O.r_of(reg, T, 0.0), rel=1e-14, abs=0.0)
    x = np.random.default_rng(3).standard_normal(shape)
    lap = _laplacian_stencil(x)
    assert np.abs(O.apply_M(kappa, x) - k0 * lap).max() <= 1e-13 * np.abs(lap).max() * k0
