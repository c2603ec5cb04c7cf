"""ctypes binding of the C oracle (test infrastructure only).

All arrays are float64 numpy arrays in C order with x fastest: a 2D image is
``(ny, nx)``, a volume ``(nz, ny, nx)``, a sinogram ``(n_angles, n_bins)``.
"""
import ctypes as C
from dataclasses import dataclass, field

import numpy as np

from .build import build as _build

REG = {"tikhonov": 0, "tv": 1, "pm_log": 2, "pm_exp": 3}
OP = {"blur": 0, "blur_mask": 1, "joseph": 2, "identity": 3}

_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(_build())
        d, i, i64, vp = C.c_double, C.c_int, C.c_int64, C.c_void_p
        P = C.POINTER
        _lib.oracle_r_of.restype = d
        _lib.oracle_r_of.argtypes = [i, d, d]
        _lib.oracle_kappa_of.restype = d
        _lib.oracle_kappa_of.argtypes = [i, d, d]
        _lib.oracle_diffusivity.restype = d
        _lib.oracle_diffusivity.argtypes = [i, P(i64), i, d, d, vp, vp]
        _lib.oracle_apply_M.argtypes = [i, P(i64), vp, vp, vp]
        _lib.oracle_mg_create.restype = vp
        _lib.oracle_mg_create.argtypes = [i, P(i64), vp, i, i, i]
        _lib.oracle_mg_free.argtypes = [vp]
        _lib.oracle_mg_apply.argtypes = [vp, vp, vp]
        _lib.oracle_mg_level_apply.argtypes = [vp, i, vp, vp]
        _lib.oracle_mg_level_size.restype = i64
        _lib.oracle_mg_level_size.argtypes = [vp, i]
        _lib.oracle_blur_taps.argtypes = [d, i, vp]
        _lib.oracle_op_data_len.restype = i64
        _lib.oracle_op_data_len.argtypes = [vp]
        _lib.oracle_apply_A.argtypes = [vp, vp, vp]
        _lib.oracle_apply_At.argtypes = [vp, vp, vp]
        _lib.oracle_mlsqr.restype = i
        _lib.oracle_mlsqr.argtypes = [vp, vp, d, i, vp, vp, vp, P(i)]
        _lib.oracle_solve.restype = i
        _lib.oracle_solve.argtypes = [vp, i, d, d, d, i, i, i, i, i, vp, vp, vp, vp, vp]
        _lib.oracle_set_kappa_rounding.argtypes = [i]
        _lib.oracle_set_kappa_rounding.restype = None
        _lib.oracle_round_bf16.argtypes = [d]
        _lib.oracle_round_bf16.restype = d
        _lib.oracle_mlsqr_s4.restype = i
        _lib.oracle_mlsqr_s4.argtypes = [vp, vp, d, i, vp, vp, vp, P(i), d]
        _lib.oracle_solve_stop.restype = i
        _lib.oracle_solve_stop.argtypes = [vp, i, d, d, d, i, i, i, i, i, d, d, vp, vp, vp, vp, vp, P(i)]
    return _lib


class _OpStruct(C.Structure):
    _fields_ = [("kind", C.c_int32), ("ndim", C.c_int32), ("n", C.c_int64 * 3),
                ("sigma", C.c_double * 3), ("radius", C.c_int32 * 3),
                ("n_angles", C.c_int32), ("n_bins", C.c_int32), ("pad_", C.c_int32),
                ("bin_spacing", C.c_double), ("mask", C.c_void_p)]


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p)


def _dims(shape):
    """numpy shape (.., ny, nx) -> (ndim, int64[3] with x first)."""
    ndim = len(shape)
    n = (C.c_int64 * 3)(*(list(reversed(shape)) + [1] * (3 - ndim)))
    return ndim, n


@dataclass
class Operator:
    """Forward map A. kind: 'blur' | 'blur_mask' | 'joseph' | 'identity'.

    shape: image shape (ny, nx) or (nz, ny, nx).  sigma/radius per axis in x, y, z order.
    mask: uint8 array of the image shape (nonzero = observed) for 'blur_mask'.
    Joseph: square image, n_angles angles a*pi/n_angles, n_bins bins of spacing bin_spacing.
    """
    kind: str
    shape: tuple
    sigma: tuple = (0.0, 0.0, 0.0)
    radius: tuple = (0, 0, 0)
    mask: np.ndarray = None
    n_angles: int = 0
    n_bins: int = 0
    bin_spacing: float = 1.0
    _s: object = field(default=None, repr=False)
    _mask_keep: object = field(default=None, repr=False)

    def struct(self):
        if self._s is None:
            s = _OpStruct()
            s.kind = OP[self.kind]
            s.ndim = len(self.shape)
            nd, n = _dims(self.shape)
            for k in range(3):
                s.n[k] = n[k]
            sg = list(self.sigma) + [0.0] * (3 - len(self.sigma))
            rd = list(self.radius) + [0] * (3 - len(self.radius))
            for k in range(3):
                s.sigma[k] = float(sg[k])
                s.radius[k] = int(rd[k])
            s.n_angles = int(self.n_angles)
            s.n_bins = int(self.n_bins)
            s.bin_spacing = float(self.bin_spacing)
            if self.mask is not None:
                self._mask_keep = np.ascontiguousarray(self.mask, dtype=np.uint8)
                s.mask = self._mask_keep.ctypes.data
            self._s = s
        return self._s

    @property
    def data_shape(self):
        if self.kind == "joseph":
            return (self.n_angles, self.n_bins)
        return tuple(self.shape)

    def A(self, x):
        x = _f64(x)
        assert x.shape == tuple(self.shape)
        y = np.empty(self.data_shape)
        lib().oracle_apply_A(C.byref(self.struct()), _ptr(x), _ptr(y))
        return y

    def At(self, y):
        y = _f64(y)
        assert y.shape == self.data_shape
        x = np.empty(self.shape)
        lib().oracle_apply_At(C.byref(self.struct()), _ptr(y), _ptr(x))
        return x


def r_of(reg, T, t):
    return lib().oracle_r_of(REG[reg], float(T), float(t))


def kappa_of(reg, T, t):
    return lib().oracle_kappa_of(REG[reg], float(T), float(t))


def blur_taps(sigma, R):
    w = np.empty(2 * R + 1)
    lib().oracle_blur_taps(float(sigma), int(R), _ptr(w))
    return w


def diffusivity(f, reg, T, kfloor=1e-4):
    """kappa_i = max(r'(t_i)/t_i, kfloor*kappa(0)) and R(f) (Algorithm 3 step 3)."""
    f = _f64(f)
    ndim, n = _dims(f.shape)
    kappa = np.empty_like(f)
    R = lib().oracle_diffusivity(ndim, n, REG[reg], float(T), float(kfloor), _ptr(f), _ptr(kappa))
    return kappa, R


def apply_M(kappa, x):
    """y = sum_d D_d^T diag(kappa) D_d x (eq. 1.13, forward differences, ghost 0)."""
    kappa, x = _f64(kappa), _f64(x)
    ndim, n = _dims(x.shape)
    y = np.empty_like(x)
    lib().oracle_apply_M(ndim, n, _ptr(kappa), _ptr(x), _ptr(y))
    return y


class Multigrid:
    """Fixed symmetric V-cycle approximation P of M^{-1} (Sec. 4.2)."""

    def __init__(self, kappa, levels, nu=2, cycles=1):
        self.kappa = _f64(kappa)
        self.shape = self.kappa.shape
        ndim, n = _dims(self.shape)
        self.h = lib().oracle_mg_create(ndim, n, _ptr(self.kappa), int(levels), int(nu), int(cycles))
        if not self.h:
            raise ValueError("multigrid setup failed (sizes not divisible or coarse operator not SPD)")
        self.levels = levels

    def apply(self, b):
        b = _f64(b)
        x = np.empty_like(b)
        lib().oracle_mg_apply(self.h, _ptr(b), _ptr(x))
        return x

    def level_size(self, l):
        return lib().oracle_mg_level_size(self.h, l)

    def level_apply(self, l, x):
        x = _f64(x)
        y = np.empty_like(x)
        lib().oracle_mg_level_apply(self.h, l, _ptr(x), _ptr(y))
        return y

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            lib().oracle_mg_free(h)
            self.h = None


def mlsqr(op: Operator, g, tau, n_inner, prec: Multigrid = None):
    """Algorithm 2 (MLSQR) from f = 0. prec None means P = I. Returns (f, rbar_hist, status)."""
    g = _f64(g)
    f = np.empty(op.shape)
    hist = np.full(n_inner, np.nan)
    st = C.c_int(0)
    done = lib().oracle_mlsqr(C.byref(op.struct()), prec.h if prec is not None else None,
                              float(tau), int(n_inner), _ptr(g), _ptr(f), _ptr(hist), C.byref(st))
    return f, hist[:done], st.value


def solve(op: Operator, g, reg, T, tau, n_outer, n_inner, levels, nu=2, cycles=1, kfloor=1e-4):
    """Algorithm 3. Returns dict(f, rbar_hist (n_outer, n_inner), R_hist, resid_hist, status)."""
    g = _f64(g)
    f = np.empty(op.shape)
    rbar = np.full((n_outer, n_inner), np.nan)
    R = np.full(n_outer + 1, np.nan)
    res = np.full(n_outer, np.nan)
    st = lib().oracle_solve(C.byref(op.struct()), REG[reg], float(T), float(tau), float(kfloor),
                            int(levels), int(nu), int(cycles), int(n_outer), int(n_inner),
                            _ptr(g), _ptr(f), _ptr(rbar), _ptr(R), _ptr(res))
    return dict(f=f, rbar_hist=rbar, R_hist=R, resid_hist=res, status=st)


__all__ = ["REG", "OP", "Operator", "Multigrid", "r_of", "kappa_of", "blur_taps",
           "diffusivity", "apply_M", "mlsqr", "solve", "lib", "mlsqr_s4", "solve_stop", "set_kappa_rounding", "round_bf16"]


def mlsqr_s4(op: Operator, g, tau, n_inner, eta_delta, prec: Multigrid = None):
    """Algorithm 2 stopped by S4 (residual estimate <= eta_delta). Returns (f, rbar_hist, status)."""
    g = _f64(g)
    f = np.empty(op.shape)
    hist = np.full(n_inner, np.nan)
    st = C.c_int(0)
    it = lib().oracle_mlsqr_s4(C.byref(op.struct()), prec.h if prec is not None else None, float(tau), int(n_inner),
                               _ptr(g), _ptr(f), _ptr(hist), C.byref(st), float(eta_delta))
    return f, hist[:it], st.value


def solve_stop(op: Operator, g, reg, T, tau, n_outer, n_inner, levels, eta_delta, r_rel, nu=2, cycles=1,
               kfloor=1e-4):
    """Algorithm 3 with S4 inner stops and the relative-R outer stop."""
    g = _f64(g)
    f = np.empty(op.shape)
    rbar = np.full((n_outer, n_inner), np.nan)
    R = np.full(n_outer + 1, np.nan)
    res = np.full(n_outer, np.nan)
    done = C.c_int(0)
    st = lib().oracle_solve_stop(C.byref(op.struct()), REG[reg], float(T), float(tau), float(kfloor), int(levels),
                                 int(nu), int(cycles), int(n_outer), int(n_inner), float(eta_delta), float(r_rel),
                                 _ptr(g), _ptr(f), _ptr(rbar), _ptr(R), _ptr(res), C.byref(done))
    return dict(f=f, rbar_hist=rbar, R_hist=R, resid_hist=res, status=st, outer_done=done.value)


def set_kappa_rounding(mode):
    """None: kappa as computed; "bf16": kappa rounded to float then bfloat16 (nearest, ties to
    even) where the diffusivity stores it, as the GPU's bfloat16-kappa variant does."""
    lib().oracle_set_kappa_rounding({None: 0, "bf16": 1}[mode])


def round_bf16(x):
    return lib().oracle_round_bf16(float(x))
