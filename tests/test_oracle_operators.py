"""Pins for the oracle's forward maps: Gaussian blur, masked blur, Joseph projector.

The paper names deblurring, inpainting and X-ray tomography as matrix-free problems
(Sec. 1); the discretisations pinned here are this project's readings (see the module
docstring of the C oracle).
"""
import numpy as np
import pytest
from scipy import ndimage

import oracle as O


def test_blur_taps_special_values():
    for sigma, R in [(2.0, 6), (4.0, 12), (0.7, 3)]:
        w = O.blur_taps(sigma, R)
        assert w.sum() == pytest.approx(1.0, abs=1e-15)
        assert np.array_equal(w, w[::-1])
        k = np.arange(-R, R + 1)
        assert np.allclose(w / w[R], np.exp(-k * k / (2 * sigma * sigma)), rtol=1e-14, atol=0)


@pytest.mark.parametrize("shape,sigma,radius", [((13, 17), (1.5, 2.5), (4, 6)),
                                                ((6, 7, 9), (1.0, 1.5, 2.0), (2, 3, 4))])
def test_blur_matches_scipy_direct_convolution(shape, sigma, radius):
    rng = np.random.default_rng(3)
    x = rng.standard_normal(shape)
    op = O.Operator("blur", shape, sigma=sigma, radius=radius)
    ws = [O.blur_taps(s, r) for s, r in zip(sigma, radius)]  # x, y(, z)
    if len(shape) == 2:
        K = np.outer(ws[1], ws[0])
    else:
        K = ws[2][:, None, None] * ws[1][None, :, None] * ws[0][None, None, :]
    ref = ndimage.convolve(x, K, mode="constant", cval=0.0)
    assert np.abs(op.A(x) - ref).max() < 1e-13


def test_blur_symmetric_adjoint_constant(dense):
    shape = (9, 11)
    op = O.Operator("blur", shape, sigma=(1.2, 2.0), radius=(3, 5))
    A = dense(op.A, shape)
    assert np.abs(A - A.T).max() < 1e-15
    At = dense(op.At, shape)
    assert np.abs(A - At).max() < 1e-15
    # taps sum to one: a constant far from the boundary is preserved
    big = O.Operator("blur", (40, 40), sigma=(2.0, 2.0), radius=(6, 6))
    y = big.A(np.ones((40, 40)))
    assert np.abs(y[6:-6, 6:-6] - 1.0).max() < 1e-14


def test_masked_blur_is_D_B(dense):
    shape = (5, 6, 7)
    rng = np.random.default_rng(4)
    mask = (rng.random(shape) > 0.3).astype(np.uint8)
    op = O.Operator("blur_mask", shape, sigma=(1.0, 1.2, 0.8), radius=(2, 3, 2), mask=mask)
    plain = O.Operator("blur", shape, sigma=(1.0, 1.2, 0.8), radius=(2, 3, 2))
    B = dense(plain.A, shape)
    D = np.diag(mask.ravel().astype(float))
    assert np.abs(dense(op.A, shape) - D @ B).max() < 1e-15
    assert np.abs(dense(op.At, shape) - B @ D).max() < 1e-15


def _joseph(n, na, nb, ds=1.0):
    return O.Operator("joseph", (n, n), n_angles=na, n_bins=nb, bin_spacing=ds)


def test_joseph_adjoint_identity():
    rng = np.random.default_rng(5)
    op = _joseph(24, 37, 35)
    x = rng.standard_normal((24, 24))
    y = rng.standard_normal((37, 35))
    Ax = op.A(x)
    lhs, rhs = float((Ax * y).sum()), float((x * op.At(y)).sum())
    assert abs(lhs - rhs) / (np.linalg.norm(Ax) * np.linalg.norm(y)) < 1e-12


def test_joseph_gaussian_blob_radon_transform():
    """Radon transform of exp(-|p-c|^2/(2a^2)) is sqrt(2 pi) a exp(-(s - c.n)^2/(2a^2))."""
    n, na, nb, a = 128, 48, 183, 8.0
    op = _joseph(n, na, nb)
    cimg = 0.5 * (n - 1)
    x0, y0 = 11.0, -17.0  # off centre: catches sign / orientation slips
    yy, xx = np.mgrid[0:n, 0:n].astype(float) - cimg
    f = np.exp(-((xx - x0) ** 2 + (yy - y0) ** 2) / (2 * a * a))
    sino = op.A(f)
    s = np.arange(nb) - 0.5 * (nb - 1)
    for ai in range(na):
        th = np.pi * ai / na
        ref = np.sqrt(2 * np.pi) * a * np.exp(-(s - (x0 * np.cos(th) + y0 * np.sin(th))) ** 2 / (2 * a * a))
        # sampling error of linear interpolation ~ (1/2)^2 / (2 a^2) of the peak
        assert np.abs(sino[ai] - ref).max() < 4e-3 * ref.max(), ai


def test_joseph_mass_and_modes():
    n, na, nb = 32, 8, 47
    op = _joseph(n, na, nb)
    rng = np.random.default_rng(6)
    f = rng.uniform(0, 1, (n, n))
    sino = op.A(f)
    # theta = 0: rays fall half way between pixel centres, every pixel counted once
    assert sino[0].sum() == pytest.approx(f.sum(), rel=1e-13)
    # theta = pi/2 (column stepping): same mass
    assert sino[na // 2].sum() == pytest.approx(f.sum(), rel=1e-12)
    # theta = 0 is a plain column sum of pairs of neighbouring columns
    colsum = f.sum(axis=0)
    k0 = int(0.5 * (nb - 1) - 0.5 * (n - 1) - 0.5)  # the ray half a pixel left of column 0
    assert sino[0][k0 - 1] == 0.0
    assert sino[0][k0] == pytest.approx(0.5 * colsum[0], rel=1e-13)
    assert sino[0][k0 + 1] == pytest.approx(0.5 * (colsum[0] + colsum[1]), rel=1e-13)


def test_identity_operator():
    x = np.arange(12.0).reshape(3, 4)
    op = O.Operator("identity", (3, 4))
    assert np.array_equal(op.A(x), x) and np.array_equal(op.At(x), x)
