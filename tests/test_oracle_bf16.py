"""The oracle's bfloat16 rounding of kappa (the storage variant of the GPU path), checked against
exact rational rounding of the single-precision value to 8 significant bits."""
from fractions import Fraction

import numpy as np
import pytest

import oracle as O


def _bf16_exact(x):
    """Nearest bfloat16 to float32(x) by exact comparison, ties to the even significand."""
    f = float(np.float32(x))
    if f == 0.0 or not np.isfinite(f):
        return f
    bits = np.array([f], dtype=np.float32).view(np.uint32)[0]
    lo_bits = bits & np.uint32(0xFFFF0000)
    lo = float(np.array([lo_bits], dtype=np.uint32).view(np.float32)[0])
    hi = float(np.array([lo_bits + np.uint32(0x10000)], dtype=np.uint32).view(np.float32)[0])
    d_lo, d_hi = abs(Fraction(f) - Fraction(lo)), abs(Fraction(hi) - Fraction(f))
    if d_lo < d_hi:
        return lo
    if d_hi < d_lo:
        return hi
    return lo if ((int(lo_bits) >> 16) & 1) == 0 else hi


def test_round_bf16_is_nearest_even():
    rng = np.random.default_rng(0)
    xs = list(rng.uniform(-1e3, 1e3, 2000)) + list(10.0 ** rng.uniform(-30, 30, 2000))
    # exact ties: a float32 whose low 16 bits are 0x8000, with even and odd kept parts
    for kept in (0x3F80, 0x3F81, 0x4000, 0x4001):
        xs.append(float(np.array([(kept << 16) | 0x8000], dtype=np.uint32).view(np.float32)[0]))
    for x in xs:
        assert O.round_bf16(x) == _bf16_exact(x), x


def test_diffusivity_with_rounding_is_the_rounded_diffusivity():
    rng = np.random.default_rng(1)
    f = rng.uniform(0, 1, (24, 20))
    k, R = O.diffusivity(f, "pm_log", 5e-2)
    O.set_kappa_rounding("bf16")
    try:
        kr, Rr = O.diffusivity(f, "pm_log", 5e-2)
    finally:
        O.set_kappa_rounding(None)
    assert Rr == R  # R(f) is not rounded
    assert np.array_equal(kr, np.array([_bf16_exact(v) for v in k.ravel()]).reshape(k.shape))
    assert np.max(np.abs(kr / k - 1)) <= 2.0 ** -8 * (1 + 1e-6)  # 8 significant bits
