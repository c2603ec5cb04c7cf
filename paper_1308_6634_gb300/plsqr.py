"""Python binding of libplsqr (include/plsqr.h): argument marshalling only.

Every computation runs in the CUDA library; this module converts torch tensors (device
memory) and numpy arrays (host memory) to pointers and checks shapes and dtypes.  The
functions keep the C names (plsqr_create, plsqr_solve, ...); ``Solver`` wraps a handle.
If the library is missing this module raises instead of falling back to anything else.
"""
import ctypes as C
import json
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libplsqr.so")

OK, E_INVALID, E_NOMEM, E_CUDA, E_BREAKDOWN, E_TIMEOUT, E_STATE = range(7)
REG = {"tikhonov": 0, "tv": 1, "pm_log": 2, "pm_exp": 3}
OP = {"blur": 0, "blur_mask": 1, "joseph": 2, "identity": 3}
PREC = {"fp64": 0, "fp32": 1}


class PlsqrError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"plsqr error {code}: {msg}")
        self.code = code


class Config(C.Structure):
    _fields_ = [("ndim", C.c_int32), ("precision", C.c_int32), ("n", C.c_int64 * 3),
                ("mg_levels", C.c_int32), ("mg_sweeps", C.c_int32), ("mg_cycles", C.c_int32),
                ("max_batch", C.c_int32), ("kappa_floor", C.c_double)]


class OperatorDesc(C.Structure):
    _fields_ = [("kind", C.c_int32), ("n_angles", C.c_int32), ("n_bins", C.c_int32), ("reserved", C.c_int32),
                ("sigma", C.c_double * 3), ("radius", C.c_int32 * 3), ("reserved2", C.c_int32),
                ("bin_spacing", C.c_double), ("mask", C.c_void_p)]


class Stats(C.Structure):
    _fields_ = [("rbar_hist", C.c_void_p), ("R_hist", C.c_void_p), ("resid_hist", C.c_void_p),
                ("status", C.c_int32), ("reserved", C.c_int32)]


_lib = None


def lib():
    """Load libplsqr.so (built by paper_1308_6634_gb300.build); raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: run `python -m paper_1308_6634_gb300.build`")
    L = C.CDLL(LIB_PATH)
    vp, i32, d, i64 = C.c_void_p, C.c_int32, C.c_double, C.c_int64
    sig = {
        "plsqr_create": ([C.POINTER(Config), vp, C.POINTER(vp)], C.c_int),
        "plsqr_set_operator": ([vp, C.POINTER(OperatorDesc)], C.c_int),
        "plsqr_solve": ([vp, vp, i32, d, d, i32, i32, vp, C.POINTER(Stats)], C.c_int),
        "plsqr_solve_host": ([vp, vp, i32, d, d, i32, i32, vp, C.POINTER(Stats)], C.c_int),
        "plsqr_solve_batch": ([vp, i32, C.POINTER(vp), C.POINTER(i32), C.POINTER(d), C.POINTER(d), i32, i32,
                               C.POINTER(vp), C.POINTER(Stats)], C.c_int),
        "plsqr_destroy": ([vp], None),
        "plsqr_last_error": ([vp], C.c_char_p),
        "plsqr_workspace_bytes": ([C.POINTER(Config), C.POINTER(OperatorDesc)], i64),
        "plsqr_apply_A": ([vp, vp, vp], C.c_int),
        "plsqr_apply_At": ([vp, vp, vp], C.c_int),
        "plsqr_diffusivity": ([vp, vp, i32, d, vp, C.POINTER(d)], C.c_int),
        "plsqr_prec_setup": ([vp, vp], C.c_int),
        "plsqr_prec_apply": ([vp, vp, vp], C.c_int),
        "plsqr_apply_M": ([vp, vp, vp], C.c_int),
        "plsqr_mlsqr": ([vp, vp, d, i32, vp, vp, C.POINTER(i32)], C.c_int),
        "plsqr_profile": ([vp, i32], C.c_int),
        "plsqr_profile_read": ([vp, vp, vp, i32], C.c_int),
        "plsqr_last_launches": ([vp], i64),
        "plsqr_check_guards": ([vp, C.POINTER(i64), C.POINTER(i64)], C.c_int),
        "plsqr_blur_noalloc": ([i32, C.POINTER(i64), i32, C.POINTER(d), C.POINTER(i32), vp, vp, vp], C.c_int),
        "plsqr_set_stopping": ([vp, i32, d, d, d], C.c_int),
        "plsqr_set_kappa_bf16": ([vp, i32], C.c_int),
        "plsqr_slot_start": ([vp, i32, vp, i32, d, d, i32, i32, C.POINTER(d)], C.c_int),
        "plsqr_step": ([vp], C.c_int),
        "plsqr_query": ([vp], C.c_int),
        "plsqr_slot_progress": ([vp, i32, C.POINTER(i32), C.POINTER(i32)], C.c_int),
        "plsqr_slot_finish": ([vp, i32, vp, C.POINTER(Stats)], C.c_int),
        "plsqr_slot_state_bytes": ([vp], i64),
        "plsqr_slot_save": ([vp, i32, vp, i64], C.c_int),
        "plsqr_slot_restore": ([vp, i32, vp, i64], C.c_int),
        "plsqr_autotune": ([vp, i32], C.c_int),
        "plsqr_mlsqr_multi_tau": ([vp, vp, i32, i32, C.POINTER(d), C.POINTER(vp), C.POINTER(d), C.POINTER(i32)],
                                  C.c_int),
        "plsqr_projected_solve": ([i32, C.POINTER(d), C.POINTER(d), d, C.POINTER(d), C.POINTER(d)], C.c_int),
        "plsqr_selftest_wait": ([i32, C.POINTER(i32)], C.c_int),
        "plsqr_set_tile_shape": ([vp, i32, i32], C.c_int),
        "plsqr_tile_shape": ([vp, i32, C.POINTER(i32), C.POINTER(i32), C.POINTER(i32), C.POINTER(i32)], C.c_int),
        "plsqr_tune_cache_export": ([C.c_char_p, i64], i64),
        "plsqr_tune_cache_import": ([C.c_char_p], i32),
        "plsqr_mg_schedule": ([vp, C.POINTER(i32), C.POINTER(i32), C.POINTER(i32)], C.c_int),
    }
    for name, (args, res) in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = res
    _lib = L
    return L


EXPORTED = ["plsqr_create", "plsqr_set_operator", "plsqr_solve", "plsqr_solve_host", "plsqr_solve_batch",
            "plsqr_destroy", "plsqr_last_error", "plsqr_workspace_bytes", "plsqr_apply_A", "plsqr_apply_At",
            "plsqr_diffusivity", "plsqr_prec_setup", "plsqr_prec_apply", "plsqr_apply_M", "plsqr_mlsqr",
            "plsqr_profile", "plsqr_profile_read", "plsqr_last_launches", "plsqr_check_guards", "plsqr_blur_noalloc",
            "plsqr_set_stopping", "plsqr_set_kappa_bf16", "plsqr_slot_start", "plsqr_step", "plsqr_query", "plsqr_slot_progress", "plsqr_slot_finish",
            "plsqr_slot_state_bytes", "plsqr_slot_save", "plsqr_slot_restore",
            "plsqr_autotune", "plsqr_set_tile_shape", "plsqr_tile_shape", "plsqr_tune_cache_export",
            "plsqr_tune_cache_import", "plsqr_mg_schedule", "plsqr_mlsqr_multi_tau",
            "plsqr_projected_solve", "plsqr_selftest_wait"]

KCLASS = ["fwd", "adj", "op_plain", "gs_fine", "mg_other", "coarse", "gk", "setup"]


def selftest_wait(complete):
    """The bounded TMA wait on a barrier that completes (returns 0) or never does (returns the
    timeout status 5); see plsqr_selftest_wait."""
    st = C.c_int32(-1)
    rc = lib().plsqr_selftest_wait(1 if complete else 0, C.byref(st))
    if rc != OK:
        raise PlsqrError(rc, "selftest_wait failed")
    return st.value


TUNE_FIELDS = ("nx", "ny", "batch", "element_size", "sweeps", "finest", "kappa_bf16", "shape")


def tune_cache_export():
    """The autotuner's process-wide tile-shape choices as text (plsqr_tune_cache_export)."""
    n = lib().plsqr_tune_cache_export(None, 0)
    buf = C.create_string_buffer(n + 1)
    lib().plsqr_tune_cache_export(buf, n + 1)
    return buf.value.decode()


def tune_cache_import(text):
    """Merge tile-shape choices (plsqr_tune_cache_import's text format); returns the entry count."""
    rc = lib().plsqr_tune_cache_import(text.encode())
    if rc < 0:
        raise PlsqrError(-rc, "malformed tile-shape cache text (nothing merged)")
    return rc


def tune_cache_json():
    """The choices as JSON: {"format": 1, "entries": [{nx, ny, batch, ..., shape}, ...]}."""
    entries = [dict(zip(TUNE_FIELDS, (int(v) for v in ln.split())))
               for ln in tune_cache_export().splitlines() if ln.strip()]
    return json.dumps({"format": 1, "entries": entries}, indent=1)


def tune_cache_load_json(text):
    d = json.loads(text)
    if d.get("format") != 1:
        raise ValueError("unknown tile-shape cache format")
    lines = "".join(" ".join(str(int(e[k])) for k in TUNE_FIELDS) + "\n" for e in d["entries"])
    return tune_cache_import(lines)


def save_tune_cache(path):
    with open(path, "w") as fh:
        fh.write(tune_cache_json())


def load_tune_cache(path):
    with open(path) as fh:
        return tune_cache_load_json(fh.read())


def projected_solve(alpha, beta, tau):
    """Host solve of the projected problem (3.6): (y, rbar history) from alpha_1..alpha_{k+1} and
    beta_1..beta_{k+1} (both of length k + 1).  Needs no GPU."""
    alpha = np.ascontiguousarray(alpha, dtype=np.float64)
    beta = np.ascontiguousarray(beta, dtype=np.float64)
    k = len(alpha) - 1
    if k < 1 or len(beta) != k + 1:
        raise ValueError("alpha and beta need k + 1 >= 2 values each")
    y = np.empty(k)
    rb = np.empty(k)
    P = C.POINTER(C.c_double)
    rc = lib().plsqr_projected_solve(k, alpha.ctypes.data_as(P), beta.ctypes.data_as(P), float(tau),
                                     y.ctypes.data_as(P), rb.ctypes.data_as(P))
    if rc != OK:
        raise PlsqrError(rc, "projected problem broke down")
    return y, rb


def _check(h, rc):
    if rc != OK and rc != E_BREAKDOWN:
        msg = lib().plsqr_last_error(h)
        raise PlsqrError(rc, msg.decode() if msg else "")
    return rc


def _torch():
    import torch
    return torch


def _dptr(t, dtype, numel=None):
    torch = _torch()
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("expected a CUDA tensor")
    if t.dtype != dtype or not t.is_contiguous():
        raise TypeError(f"expected a contiguous {dtype} tensor, got {t.dtype}")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"expected {numel} elements, got {t.numel()}")
    return C.c_void_p(t.data_ptr())


def make_config(shape, precision="fp32", levels=1, sweeps=2, cycles=1, max_batch=1, kappa_floor=1e-4):
    """shape: (ny, nx) or (nz, ny, nx)."""
    c = Config()
    c.ndim = len(shape)
    c.precision = PREC[precision]
    dims = list(reversed(shape)) + [1] * (3 - len(shape))
    for k in range(3):
        c.n[k] = int(dims[k])
    c.mg_levels, c.mg_sweeps, c.mg_cycles = int(levels), int(sweeps), int(cycles)
    c.max_batch = int(max_batch)
    c.kappa_floor = float(kappa_floor)
    return c


def make_operator(kind, sigma=(0, 0, 0), radius=(0, 0, 0), mask=None, n_angles=0, n_bins=0, bin_spacing=1.0):
    o = OperatorDesc()
    o.kind = OP[kind]
    sg = list(sigma) + [0.0] * (3 - len(sigma))
    rd = list(radius) + [0] * (3 - len(radius))
    for k in range(3):
        o.sigma[k] = float(sg[k])
        o.radius[k] = int(rd[k])
    o.n_angles, o.n_bins, o.bin_spacing = int(n_angles), int(n_bins), float(bin_spacing)
    o.mask = C.c_void_p(mask.data_ptr()) if mask is not None else None
    return o


def plsqr_create(config, stream=None):
    h = C.c_void_p()
    rc = lib().plsqr_create(C.byref(config), C.c_void_p(stream or 0), C.byref(h))
    if rc != OK:
        raise PlsqrError(rc, "plsqr_create failed")
    return h


def plsqr_workspace_bytes(config, op=None):
    return lib().plsqr_workspace_bytes(C.byref(config), C.byref(op) if op is not None else None)


def plsqr_blur_noalloc(x, sigma, radius, y=None, stream=None):
    """y = B x for a contiguous float32/float64 CUDA tensor of shape (ny, nx) or (nz, ny, nx),
    without any device allocation inside the library (sigma, radius in x, y(, z) order)."""
    torch = _torch()
    if not isinstance(x, torch.Tensor) or x.dtype not in (torch.float32, torch.float64):
        raise TypeError(f"plsqr_blur_noalloc: x must be a float32 or float64 tensor, got {getattr(x, 'dtype', x)}")
    if y is None:
        y = torch.empty_like(x)
    if not isinstance(y, torch.Tensor) or y.dtype != x.dtype:
        raise TypeError(f"plsqr_blur_noalloc: y must have x's dtype {x.dtype}")
    prec = PREC["fp64"] if x.dtype == torch.float64 else PREC["fp32"]
    nd = x.dim()
    dims = list(reversed(x.shape)) + [1] * (3 - nd)
    n = (C.c_int64 * 3)(*[int(v) for v in dims])
    sg = (C.c_double * 3)(*(list(map(float, sigma)) + [0.0] * (3 - len(sigma))))
    rd = (C.c_int32 * 3)(*(list(map(int, radius)) + [0] * (3 - len(radius))))
    rc = lib().plsqr_blur_noalloc(nd, n, prec, sg, rd, _dptr(x, x.dtype), _dptr(y, x.dtype, x.numel()),
                                  C.c_void_p(stream if stream is not None else _current_stream()))
    if rc != OK:
        raise PlsqrError(rc, "plsqr_blur_noalloc failed")
    return y


def _current_stream():
    torch = _torch()
    return torch.cuda.current_stream().cuda_stream


class Solver:
    """One handle: a problem size, a forward map and the priorconditioner shape."""

    def __init__(self, shape, precision="fp32", levels=1, sweeps=2, cycles=1, max_batch=1, kappa_floor=1e-4,
                 stream=None):
        torch = _torch()
        self.shape = tuple(int(s) for s in shape)
        self.N = int(np.prod(self.shape))
        self.precision = precision
        self.dtype = torch.float64 if precision == "fp64" else torch.float32
        self.np_dtype = np.float64 if precision == "fp64" else np.float32
        self.config = make_config(self.shape, precision, levels, sweeps, cycles, max_batch, kappa_floor)
        self.max_batch = max_batch
        self.h = plsqr_create(self.config, stream if stream is not None else _current_stream())
        self.data_shape = self.shape
        self._mask = None
        self._slot_shape = {}  # slot -> (n_outer, n_inner) given at slot_start

    def close(self):
        if getattr(self, "h", None):
            lib().plsqr_destroy(self.h)
            self.h = None

    __del__ = close

    @property
    def m(self):
        return int(np.prod(self.data_shape))

    def set_operator(self, kind, sigma=(0, 0, 0), radius=(0, 0, 0), mask=None, n_angles=0, n_bins=0,
                     bin_spacing=1.0):
        torch = _torch()
        if mask is not None:
            mask = torch.as_tensor(np.ascontiguousarray(mask, dtype=np.uint8)).cuda() \
                if not isinstance(mask, torch.Tensor) else mask.to(torch.uint8).contiguous().cuda()
            self._mask = mask
        o = make_operator(kind, sigma, radius, mask, n_angles, n_bins, bin_spacing)
        _check(self.h, lib().plsqr_set_operator(self.h, C.byref(o)))
        self.data_shape = (n_angles, n_bins) if kind == "joseph" else self.shape
        return self

    def _stats(self, n_outer, n_inner):
        rbar = np.full((n_outer, n_inner), np.nan)
        R = np.full(n_outer + 1, np.nan)
        res = np.full(n_outer, np.nan)
        st = Stats(rbar.ctypes.data, R.ctypes.data, res.ctypes.data, 0, 0)
        return st, dict(rbar_hist=rbar, R_hist=R, resid_hist=res)

    def solve(self, g, reg, T, tau, n_outer, n_inner, f_out=None, stats=True):
        """Algorithm 3 on device data g; returns (f, info dict or None)."""
        torch = _torch()
        if f_out is None:
            f_out = torch.empty(self.shape, dtype=self.dtype, device=g.device)
        gp = _dptr(g, self.dtype, self.m)
        fp = _dptr(f_out, self.dtype, self.N)
        if stats:
            st, info = self._stats(n_outer, n_inner)
            rc = _check(self.h, lib().plsqr_solve(self.h, gp, REG[reg], float(T), float(tau), int(n_outer),
                                                  int(n_inner), fp, C.byref(st)))
            info["status"] = rc
            return f_out, info
        _check(self.h, lib().plsqr_solve(self.h, gp, REG[reg], float(T), float(tau), int(n_outer), int(n_inner),
                                          fp, None))
        return f_out, None

    def solve_host(self, g, reg, T, tau, n_outer, n_inner, f_out=None, stats=False):
        """Algorithm 3 on host data (numpy, ideally pinned); copies are part of the call."""
        g = np.ascontiguousarray(g, dtype=self.np_dtype) if isinstance(g, np.ndarray) else g
        if f_out is None:
            f_out = np.empty(self.shape, dtype=self.np_dtype)
        gp = C.c_void_p(g.ctypes.data if isinstance(g, np.ndarray) else g.data_ptr())
        fp = C.c_void_p(f_out.ctypes.data if isinstance(f_out, np.ndarray) else f_out.data_ptr())
        st, info = (self._stats(n_outer, n_inner) if stats else (None, None))
        rc = _check(self.h, lib().plsqr_solve_host(self.h, gp, REG[reg], float(T), float(tau), int(n_outer),
                                                   int(n_inner), fp, C.byref(st) if stats else None))
        if info is not None:
            info["status"] = rc
        return f_out, info

    def solve_batch(self, gs, regs, Ts, taus, n_outer, n_inner, f_outs=None, stats=True):
        torch = _torch()
        count = len(gs)
        if f_outs is None:
            f_outs = [torch.empty(self.shape, dtype=self.dtype, device=gs[0].device) for _ in range(count)]
        garr = (C.c_void_p * count)(*[_dptr(g, self.dtype, self.m).value for g in gs])
        farr = (C.c_void_p * count)(*[_dptr(f, self.dtype, self.N).value for f in f_outs])
        rarr = (C.c_int32 * count)(*[REG[r] for r in regs])
        tarr = (C.c_double * count)(*[float(t) for t in Ts])
        uarr = (C.c_double * count)(*[float(t) for t in taus])
        infos = None
        sarr = None
        if stats:
            pairs = [self._stats(n_outer, n_inner) for _ in range(count)]
            sarr = (Stats * count)(*[p[0] for p in pairs])
            infos = [p[1] for p in pairs]
        rc = _check(self.h, lib().plsqr_solve_batch(self.h, count, garr, rarr, tarr, uarr, int(n_outer),
                                                    int(n_inner), farr, sarr))
        if infos is not None:
            for k, inf in enumerate(infos):
                inf["status"] = sarr[k].status
            return f_outs, infos
        return f_outs, None

    # ---- instrumentation ----
    def profile(self, enable=True):
        _check(self.h, lib().plsqr_profile(self.h, 1 if enable else 0))

    def profile_read(self):
        ms = (C.c_double * len(KCLASS))()
        cnt = (C.c_int64 * len(KCLASS))()
        _check(self.h, lib().plsqr_profile_read(self.h, ms, cnt, len(KCLASS)))
        return {k: (ms[i], cnt[i]) for i, k in enumerate(KCLASS)}

    def last_launches(self):
        return int(lib().plsqr_last_launches(self.h))

    def check_guards(self):
        """(allocations with guard bands, allocations whose bands changed); bands exist when
        PLSQR_GUARD=1 was set as the handle was created."""
        checked, bad = C.c_int64(0), C.c_int64(0)
        _check(self.h, lib().plsqr_check_guards(self.h, C.byref(checked), C.byref(bad)))
        return checked.value, bad.value

    def set_stopping(self, eta=0.0, delta=0.0, r_rel=0.0, index=-1):
        """S4 with eta * delta (0: off) and the outer stop on a relative R decrease below r_rel
        (0: off) for later solves; index -1 = every instance."""
        _check(self.h, lib().plsqr_set_stopping(self.h, int(index), float(eta), float(delta), float(r_rel)))

    def set_kappa_bf16(self, on=True):
        """Keep kappa in bfloat16 for later solves (2D single precision, temporally blocked V-cycle)."""
        _check(self.h, lib().plsqr_set_kappa_bf16(self.h, 1 if on else 0))

    def mlsqr_multi_tau(self, g, taus, n_inner):
        """One MLSQR bidiagonalisation from f = 0 with the current hierarchy, its Lanczos vectors
        stored; returns ([f(tau) for tau in taus], rbar histories (len(taus) x n_inner), steps done)."""
        torch = _torch()
        taus = [float(t) for t in taus]
        fs = [torch.empty(self.shape, dtype=self.dtype, device=g.device) for _ in taus]
        ta = (C.c_double * len(taus))(*taus)
        fp = (C.c_void_p * len(taus))(*[_dptr(f, self.dtype, self.N) for f in fs])
        hist = (C.c_double * (len(taus) * n_inner))()
        done = C.c_int32(0)
        _check(self.h, lib().plsqr_mlsqr_multi_tau(self.h, _dptr(g, self.dtype, self.m), int(n_inner), len(taus), ta,
                                                   fp, hist, C.byref(done)))
        return fs, np.array(hist[:], dtype=np.float64).reshape(len(taus), n_inner), done.value

    # ---- V-cycle tile shapes ----
    def autotune(self, fresh=False):
        """Time every compiled tile shape on each 2D V-cycle level and keep the fastest."""
        _check(self.h, lib().plsqr_autotune(self.h, 1 if fresh else 0))

    def set_tile_shape(self, level, shape):
        _check(self.h, lib().plsqr_set_tile_shape(self.h, int(level), int(shape)))

    def tile_shape(self, level):
        """(shape id, tile x, tile y, threads) of a level; id -1 where the tiled 2D kernels do not run."""
        v = [C.c_int32() for _ in range(4)]
        _check(self.h, lib().plsqr_tile_shape(self.h, int(level), *[C.byref(x) for x in v]))
        return tuple(x.value for x in v)

    def mg_schedule(self, detail=False):
        """1: the 2D V-cycle runs (from some level down) as one cooperative launch; 0: per-level
        launches; -1: not chosen yet.  detail=True: (that, first level, block cap)
        (plsqr_mg_schedule)."""
        v = [C.c_int32() for _ in range(3)]
        _check(self.h, lib().plsqr_mg_schedule(self.h, *[C.byref(x) for x in v]))
        return tuple(x.value for x in v) if detail else v[0].value

    # ---- slots (continuous batching) ----
    def slot_start(self, slot, g, reg, T, tau, n_outer, n_inner, sigma=None):
        sg = None if sigma is None else (C.c_double * 2)(*[float(x) for x in sigma])
        _check(self.h, lib().plsqr_slot_start(self.h, int(slot), _dptr(g, self.dtype, self.m), REG[reg], float(T),
                                              float(tau), int(n_outer), int(n_inner), sg))
        self._slot_shape[int(slot)] = (int(n_outer), int(n_inner))

    def step(self):
        _check(self.h, lib().plsqr_step(self.h))

    def busy(self):
        rc = lib().plsqr_query(self.h)
        if rc < 0:
            _check(self.h, -rc)
        return rc == 1

    def slot_progress(self, slot):
        """(outer steps done, state): state 0 empty, 1 running, 2 stopped early by the outer rule."""
        done, act = C.c_int32(0), C.c_int32(0)
        _check(self.h, lib().plsqr_slot_progress(self.h, int(slot), C.byref(done), C.byref(act)))
        return done.value, act.value

    def slot_finish(self, slot, n_outer, n_inner, f_out=None):
        """Returns (f, info) for a slot started for n_outer steps of n_inner iterations (the
        history arrays are sized by the values given at slot_start, which must match)."""
        torch = _torch()
        shape = self._slot_shape.get(int(slot))
        if shape is not None and shape != (int(n_outer), int(n_inner)):
            raise ValueError(f"slot {slot} was started for {shape[0]} x {shape[1]} iterations")
        if f_out is None:
            f_out = torch.empty(self.shape, dtype=self.dtype, device=torch.device("cuda", torch.cuda.current_device()))
        st, info = self._stats(*(shape or (n_outer, n_inner)))
        rc = _check(self.h, lib().plsqr_slot_finish(self.h, int(slot), _dptr(f_out, self.dtype, self.N),
                                                    C.byref(st)))
        self._slot_shape.pop(int(slot), None)
        info["status"] = rc
        return f_out, info

    def slot_save(self, slot):
        """The checkpoint of running `slot` at its current outer-step boundary (bytes; see
        plsqr_slot_save).  The slot keeps running."""
        n = int(lib().plsqr_slot_state_bytes(self.h))
        if n < 0:
            raise PlsqrError(E_STATE, "the handle is not in slot mode")
        buf = (C.c_char * n)()
        _check(self.h, lib().plsqr_slot_save(self.h, int(slot), buf, n))
        return bytes(buf)

    def slot_restore(self, slot, data, n_outer, n_inner):
        """Starts `slot` from a checkpoint of slot_save (of a request started for n_outer steps of
        n_inner iterations); it continues under step() and ends with slot_finish."""
        buf = (C.c_char * len(data)).from_buffer_copy(data)
        _check(self.h, lib().plsqr_slot_restore(self.h, int(slot), buf, len(data)))
        self._slot_shape[int(slot)] = (int(n_outer), int(n_inner))

    # ---- single steps ----
    def apply_A(self, x, y=None):
        torch = _torch()
        y = torch.empty(self.data_shape, dtype=self.dtype, device=x.device) if y is None else y
        _check(self.h, lib().plsqr_apply_A(self.h, _dptr(x, self.dtype, self.N), _dptr(y, self.dtype, self.m)))
        return y

    def apply_At(self, y, x=None):
        torch = _torch()
        x = torch.empty(self.shape, dtype=self.dtype, device=y.device) if x is None else x
        _check(self.h, lib().plsqr_apply_At(self.h, _dptr(y, self.dtype, self.m), _dptr(x, self.dtype, self.N)))
        return x

    def diffusivity(self, f, reg, T):
        torch = _torch()
        kappa = torch.empty(self.shape, dtype=self.dtype, device=f.device)
        R = C.c_double(0.0)
        _check(self.h, lib().plsqr_diffusivity(self.h, _dptr(f, self.dtype, self.N), REG[reg], float(T),
                                               _dptr(kappa, self.dtype, self.N), C.byref(R)))
        return kappa, R.value

    def prec_setup(self, kappa):
        _check(self.h, lib().plsqr_prec_setup(self.h, _dptr(kappa, self.dtype, self.N)))

    def prec_apply(self, b, x=None):
        torch = _torch()
        x = torch.empty(self.shape, dtype=self.dtype, device=b.device) if x is None else x
        _check(self.h, lib().plsqr_prec_apply(self.h, _dptr(b, self.dtype, self.N), _dptr(x, self.dtype, self.N)))
        return x

    def apply_M(self, x, y=None):
        torch = _torch()
        y = torch.empty(self.shape, dtype=self.dtype, device=x.device) if y is None else y
        _check(self.h, lib().plsqr_apply_M(self.h, _dptr(x, self.dtype, self.N), _dptr(y, self.dtype, self.N)))
        return y

    def mlsqr(self, g, tau, n_inner):
        torch = _torch()
        f = torch.empty(self.shape, dtype=self.dtype, device=g.device)
        hist = np.full(n_inner, np.nan)
        it = C.c_int32(0)
        rc = _check(self.h, lib().plsqr_mlsqr(self.h, _dptr(g, self.dtype, self.m), float(tau), int(n_inner),
                                              _dptr(f, self.dtype, self.N), C.c_void_p(hist.ctypes.data),
                                              C.byref(it)))
        return f, hist[:it.value], rc
