"""Continuous-batching serving loop for deblurring and tomography solves.

Requests (a blur or Joseph forward map, an image size, a regulariser, data g) are grouped into
buckets that share one library handle: the same image size and operator class.  A blur bucket
holds one register-blocked radius class (6, 9, 12 or 15) and gives every slot its own sigma
(plsqr_slot_start's per-slot taps), so requests with different blur widths run in one launch; a
tomography bucket holds one angle count.  Each handle's max_batch instances are slots.  A
bucket advances all its running slots one lagged-diffusivity step (Algorithm 3, steps 3-5) per
plsqr_step, asynchronously on the handle's own stream, so the buckets' work overlaps on the
device; between steps finished requests leave and queued ones enter (continuous batching).  The
iterates and Krylov state of a request stay on the device from admission to completion.
Buckets are created while the device-memory budget (plsqr_workspace_bytes of each handle)
allows; requests for a bucket that cannot be created wait until an idle bucket is released.

Requests use 10 x 30 iterations, T = 1e-2 (TV) or 5e-2 (Perona-Malik, log form), tau = 1e-3,
a V-cycle down to at most 16 cells per axis, and ceil(n sqrt 2) (made odd) detector bins.
"""
import collections
import math
import os
import time
from dataclasses import dataclass, field

import numpy as np

from . import plsqr, synth

SIZES = (128, 256, 512, 1024)
SIZE_P = (0.4, 0.3, 0.2, 0.1)
ANGLES = (180, 240, 300, 360)
R_CLASSES = (6, 9, 12, 15)
T_OF = {"tv": 1e-2, "pm_log": 5e-2}


@dataclass
class Request:
    rid: int
    kind: str              # "blur" or "joseph"
    n: int                 # image is n x n
    reg: str
    T: float
    tau: float
    n_outer: int
    n_inner: int
    seed: int
    t_arrival: float = 0.0  # seconds after the stream starts
    sigma: float = 0.0      # blur
    n_angles: int = 0       # tomography
    # stopping rules (0: off): S4 with eta * delta per inner solve, the outer stop when R falls by
    # less than r_rel; a request stopped by the outer rule leaves its slot early
    eta: float = 0.0
    delta: float = 0.0
    r_rel: float = 0.0
    # filled by the engine
    t_admit: float = math.nan
    t_done: float = math.nan
    bucket: tuple = ()
    status: int = -1


def levels_for(n):
    """Coarsen by 2 until at most 16 cells per axis."""
    L = 1
    while n % 2 == 0 and n // 2 >= 16 and n > 16:
        n //= 2
        L += 1
    return L


def n_bins_for(n):
    b = int(math.ceil(n * math.sqrt(2.0)))
    return b if b % 2 else b + 1


def r_class(sigma):
    r = int(math.ceil(3.0 * sigma))
    for c in R_CLASSES:
        if r <= c:
            return c
    raise ValueError("sigma too large for the blur radius classes")


def bucket_key(req):
    return ("blur", req.n, r_class(req.sigma)) if req.kind == "blur" else ("joseph", req.n, req.n_angles)


def make_stream(count, rate, seed=0, n_outer=10, n_inner=30, sizes=SIZES, size_p=SIZE_P, angles=ANGLES):
    """Seeded request stream with Poisson arrivals at `rate` per second: half deblurring (sigma
    uniform in [1.5, 5]), half tomography; sizes, regularisers and seeds drawn independently."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for k in range(count):
        t += rng.exponential(1.0 / rate)
        kind = "blur" if rng.random() < 0.5 else "joseph"
        n = int(rng.choice(sizes, p=size_p))
        reg = "tv" if rng.random() < 0.5 else "pm_log"
        r = Request(rid=k, kind=kind, n=n, reg=reg, T=T_OF[reg], tau=1e-3, n_outer=n_outer, n_inner=n_inner,
                    seed=int(rng.integers(1 << 30)), t_arrival=t)
        if kind == "blur":
            r.sigma = float(rng.uniform(1.5, 5.0))
        else:
            r.n_angles = int(rng.choice(angles))
        out.append(r)
    return out


def _bucket_solver(key, slots, torch):
    kind, n, p = key
    S = plsqr.Solver((n, n), "fp32", levels=levels_for(n), sweeps=2, cycles=1, max_batch=slots)
    if kind == "blur":
        S.set_operator("blur", sigma=(p / 3.0, p / 3.0), radius=(p, p))
    else:
        S.set_operator("joseph", n_angles=p, n_bins=n_bins_for(n))
    return S


def bucket_bytes(key, slots):
    kind, n, p = key
    cfg = plsqr.make_config((n, n), "fp32", levels_for(n), 2, 1, slots)
    op = (plsqr.make_operator("blur", sigma=(p / 3.0, p / 3.0), radius=(p, p)) if kind == "blur"
          else plsqr.make_operator("joseph", n_angles=p, n_bins=n_bins_for(n)))
    return int(plsqr.plsqr_workspace_bytes(cfg, op))


_PROJ = {}


def make_data(req, torch, dev):
    """g = A f_true + 1% noise for a request (device, float32).  Blur data come from the
    library's allocation-free blur with the request's own sigma; tomography data from a
    one-instance handle with the request's geometry."""
    n = req.n
    if req.kind == "blur":
        f = synth.phantom_rects_disks(n, max(6, n // 25), max(4, n // 40), req.seed)
        r = int(math.ceil(3.0 * req.sigma))
        Af = plsqr.plsqr_blur_noalloc(torch.as_tensor(f, dtype=torch.float32, device=dev), (req.sigma, req.sigma),
                                      (r, r))
    else:
        f = synth.phantom_ellipses(n, max(5, n // 40), req.seed)
        key = (n, req.n_angles)
        if key not in _PROJ:
            P = plsqr.Solver((n, n), "fp32", levels=levels_for(n))
            P.set_operator("joseph", n_angles=req.n_angles, n_bins=n_bins_for(n))
            _PROJ[key] = P
        Af = _PROJ[key].apply_A(torch.as_tensor(f, dtype=torch.float32, device=dev))
    z = synth.standard_noise(tuple(Af.shape), req.seed + 104729)
    sig = 0.01 * float(torch.linalg.vector_norm(Af.double())) / math.sqrt(Af.numel())
    return (Af.double() + sig * torch.as_tensor(z, device=dev)).float().contiguous(), f


class Bucket:
    def __init__(self, key, slots, torch):
        self.key = key
        self.slots = slots
        self.solver = _bucket_solver(key, slots, torch)
        self.running = {}                 # slot -> (Request, g tensor)
        self.queue = collections.deque()  # (Request, g tensor)
        self.results = {}
        self.steps = 0
        self.last_used = time.perf_counter()

    def idle(self):
        return not self.running and not self.queue

    def tick(self, now_fn, keep_results):
        """Between steps: collect finished slots, admit queued requests, launch the next step.
        Returns the number of requests completed."""
        S = self.solver
        if S.busy():
            return 0
        done = 0
        for slot, (req, _) in list(self.running.items()):
            k, state = S.slot_progress(slot)
            if k >= req.n_outer or state == 2:
                f, info = S.slot_finish(slot, req.n_outer, req.n_inner)
                req.t_done = now_fn()
                req.status = info["status"]
                if keep_results:
                    self.results[req.rid] = (f, info)
                del self.running[slot]
                done += 1
        free = [s for s in range(self.slots) if s not in self.running]
        while free and self.queue:
            req, g = self.queue.popleft()
            slot = free.pop(0)
            S.set_stopping(req.eta, req.delta, req.r_rel, index=slot)
            S.slot_start(slot, g, req.reg, req.T, req.tau, req.n_outer, req.n_inner,
                         sigma=(req.sigma, req.sigma) if req.kind == "blur" else None)
            req.t_admit = now_fn()
            self.running[slot] = (req, g)
        if self.running:
            S.step()
            self.steps += 1
            self.last_used = time.perf_counter()
        return done


class Engine:
    """Admission by a device-memory budget; one bucket (handle, stream, slots) per operator class."""

    def __init__(self, hbm_budget_bytes=40 << 30, slots_for_size=None, keep_results=False, tune_cache=None):
        """tune_cache: a JSON file of tile-shape choices (plsqr.save_tune_cache).  If it exists it
        is loaded, so that the first step of each bucket skips the timing; save_tune_cache()
        writes the choices back."""
        import torch
        self.torch = torch
        self.budget = int(hbm_budget_bytes)
        self.slots_for_size = slots_for_size or {128: 16, 256: 8, 512: 4, 1024: 2}
        self.buckets = {}
        self.bytes_used = 0
        self.keep_results = keep_results
        self.refused = 0
        self.tune_cache = tune_cache
        if tune_cache and os.path.exists(tune_cache):
            plsqr.load_tune_cache(tune_cache)

    def save_tune_cache(self):
        if self.tune_cache:
            plsqr.save_tune_cache(self.tune_cache)

    def slots_of(self, n):
        return self.slots_for_size.get(n, 4)

    def bucket(self, key, create=True):
        b = self.buckets.get(key)
        if b is not None or not create:
            return b
        need = bucket_bytes(key, self.slots_of(key[1]))
        while self.bytes_used + need > self.budget:
            idle = [k for k, v in self.buckets.items() if v.idle()]
            if not idle:
                self.refused += 1
                return None
            victim = min(idle, key=lambda k: self.buckets[k].last_used)
            self.release(victim)
        b = Bucket(key, self.slots_of(key[1]), self.torch)
        b.bytes = need
        self.buckets[key] = b
        self.bytes_used += need
        return b

    def release(self, key):
        b = self.buckets.pop(key)
        self.bytes_used -= b.bytes
        del b

    def run(self, requests, data, realtime=True, t_limit=600.0):
        """Serve `requests` (sorted by arrival) with device data `data[rid]`; arrivals follow
        t_arrival in wall-clock time when realtime.  Returns the requests, timed."""
        pending = collections.deque(sorted(requests, key=lambda r: r.t_arrival))
        waiting = collections.deque()   # arrived, bucket not yet available
        t0 = time.perf_counter()
        now = lambda: time.perf_counter() - t0
        total, done = len(requests), 0
        while done < total:
            t = now()
            if t > t_limit:
                raise RuntimeError(f"serving run exceeded {t_limit} s ({done}/{total} done)")
            while pending and (not realtime or pending[0].t_arrival <= t):
                waiting.append(pending.popleft())
            for _ in range(len(waiting)):
                req = waiting.popleft()
                key = bucket_key(req)
                b = self.bucket(key)
                if b is None:
                    waiting.append(req)
                    continue
                req.bucket = key
                b.queue.append((req, data[req.rid]))
            progressed = 0
            for b in list(self.buckets.values()):
                got = b.tick(now, self.keep_results)
                done += got
                progressed += got
            if not progressed:
                time.sleep(0.0002)
        return requests

    def results(self):
        out = {}
        for b in self.buckets.values():
            out.update(b.results)
        return out


def summarize(requests):
    lat = np.array([1e3 * (r.t_done - r.t_arrival) for r in requests])
    wait = np.array([1e3 * (r.t_admit - r.t_arrival) for r in requests])
    t_first = min(r.t_arrival for r in requests)
    t_last = max(r.t_done for r in requests)
    by_kind = collections.Counter(r.kind for r in requests)
    return {"solves_per_s": len(requests) / (t_last - t_first), "p50_ms": float(np.percentile(lat, 50)),
            "p99_ms": float(np.percentile(lat, 99)), "mean_ms": float(lat.mean()),
            "queue_wait_p50_ms": float(np.percentile(wait, 50)), "queue_wait_p99_ms": float(np.percentile(wait, 99)),
            "requests": len(requests), "by_kind": dict(by_kind),
            "breakdowns": int(sum(1 for r in requests if r.status not in (0,)))}
