"""Benchmark: solves/s of the priorconditioned lagged-diffusivity solver on one workload.

One step = one batch of B complete solves (Algorithm 3: n_outer lagged-diffusivity steps,
each with n_inner MLSQR iterations and a fresh V-cycle priorconditioner) of the 1024x1024
FP32 deblurring workload (Gaussian blur sigma 4 truncated at radius 12, 1% noise,
Perona-Malik log regulariser T = 5e-2, tau = 1e-3, 15 x 50 iterations, 6-level V-cycle with
2 red-black sweeps per side), inputs resident in device memory.  Multi-GPU runs are replicas
(independent instances per rank, no collective on the data path; weak scaling).

JSON line keys beyond the base contract: p50_ms/p99_ms (per-step latency), roofline of the
dominant kernel class (eager profiling pass with CUDA events on the launch stream), e2e (host
buffers, copies inside the timed region), clocks (nvidia-smi sampled during the timed region),
fp64_single (the plain double-precision single-instance form), workloads (the 192^3 inpainting,
512^2 tomography x1 and x32 and the serving stream, each with its own value, p50/p99, roofline
and clocks), and the oracle leg: cpu_baseline (the FP64 CPU oracle timed on one whole outer step
of the workload, on one core and on all cores at once; a solve is n_outer such steps) and
accuracy (the GPU results of the whole n_outer x n_inner solve against a whole oracle solve of
the same data, beside the oracle's own spread under a 1e-16 perturbation of g).

--impl reference times the FP64 CPU oracle itself on the same workload and metric: each step
is one outer step of the workload on every host core at once.
"""
import argparse
import hashlib
import re
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

L2_BYTES = 126 * 1024 * 1024
METRIC = "solves/s and p50/p99 ms at <=1e-4 rel err vs FP64 oracle; HBM GB/s vs peak"

# Algorithmic bytes per instance and per launch of each kernel class, in units of
# (vector element size x N): the minimum reads and writes each pass forces, for the kernels the
# 2D single-precision blur workload runs.
#   fwd:  first iteration v~ in, u_prev in, u out (3); later iterations also apply the previous
#         iteration's update on the same cells: + w~, f in and out (7)      -> (3 + 7 (n-1)) / n
#   adj:  u in, p~ in, p~ out                                               3
#   gs_fine (finest-level V-cycle launches, pre and post alternate):
#         pre:  p~ (rhs), kappa in, x out, restricted residual out (1/4)    3.25
#         post: x_in, p~, kappa, coarse correction (1/4) in, v~ out         4.25  -> mean 3.75
# FP32 FMA lanes x SMs x maximum SM clock of the GB300 (152 SMs, 128 FP32 lanes each, 2070 MHz):
# the peak the Joseph projector, a gather- and issue-bound kernel, is measured against
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12


def joseph_samples(n, n_angles, n_bins, spacing=1.0):
    """Interpolation samples of one Joseph forward apply: for each ray, the rows (near-vertical rays)
    or columns it steps over where the sample falls inside the image (pixel centres at
    j - (n-1)/2, bins at (k - (n_b-1)/2) * spacing, angles a pi / n_angles).  Each sample is two
    gathers and two FMA."""
    c = (n - 1) / 2.0
    s = (np.arange(n_bins) - (n_bins - 1) / 2.0) * spacing
    steps = np.arange(n) - c
    total = 0
    for a in range(n_angles):
        th = a * np.pi / n_angles
        ct, st = np.cos(th), np.sin(th)
        if 4 * a < n_angles or 4 * a > 3 * n_angles:
            pos = (s[None, :] - steps[:, None] * st) / ct   # x at each row
        else:
            pos = (s[None, :] - steps[:, None] * ct) / st   # y at each column
        total += int(np.count_nonzero(np.abs(pos) <= c))
    return total


def alg_units(W, kappa_bf16=False):
    """Algorithmic bytes per launch of each roofline class, in units of (element size x cells x
    instances): the minimum reads and writes of one pass.  2D V-cycle, finest level (mean of the
    pre- and post-smoothing launches): pre reads b and kappa and writes x and the restricted
    residual (1/4); post reads x_in, b, kappa and the coarse correction (1/4) and writes x.
    kappa in bfloat16 counts half."""
    n = W.n_inner
    two_d_blur = W.kind in ("blur", "blur_mask") and len(W.shape) == 2
    fused_update = two_d_blur and W.precision == "fp32" and W.radius[0] == W.radius[1] and W.radius[0] in (6, 9, 12, 15)
    fwd = (3.0 + 7.0 * (n - 1)) / n if fused_update else 3.0
    if len(W.shape) == 2:
        k = 0.5 if kappa_bf16 else 1.0
        return {"fwd": fwd, "adj": 3.0, "gs_fine": ((2.25 + k) + (3.25 + k)) / 2}
    # 3D: one launch per red-black half sweep: x of the other colour (1/2), kappa (1),
    # b of this colour (1/2) in, x of this colour (1/2) out
    return {"fwd": fwd, "adj": 3.0, "gs_fine": 2.5}


def beyond_alg_units(W):
    """Bytes per launch that a class moves beyond its algorithmic ones, same units: the 2D
    V-cycle kernels also read the reciprocal diagonal of the level (formed once per outer step,
    a trade of one plane of reads for the division of every sweep)."""
    return {"gs_fine": 1.0} if len(W.shape) == 2 else {}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--batch", type=int, default=1)
    ap.add_argument("--workload", default="deblur1024_fp32")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-profile", action="store_true")
    ap.add_argument("--no-fp64-single", action="store_true")
    ap.add_argument("--kappa-bf16", action="store_true", help="keep kappa in bfloat16 (2D single precision)")
    ap.add_argument("--tiles", default=None,
                    help="V-cycle tile shape id per level (comma-separated) instead of the autotuner's choice")
    ap.add_argument("--rate", type=float, default=200.0, help="serving: arrivals per second")
    ap.add_argument("--requests", type=int, default=2000, help="serving: requests in the stream")
    ap.add_argument("--hbm-budget-gb", type=float, default=40.0, help="serving: device-memory budget")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the other workloads (192^3 inpainting, 512^2 tomography x1 and x32, serving)")
    ap.add_argument("--no-accuracy", action="store_true", help="skip the whole-solve accuracy against the oracle")
    ap.add_argument("--cpu-procs", type=int, default=0,
                    help="oracle processes at once for the all-cores figures (0: every usable core, at most 32)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        return float(d.get("hbm_gbs", 6800.0)), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi samples (200 ms) during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm)}


# the sources that define the kernels of the roofline classes (blur, V-cycle) and their device
# helpers; the launcher declarations in kernels.cuh are left out
TRAFFIC_SOURCES = ("common.cuh", "tma.cuh", "k_ops.cu", "k_mg.cu", "k_mg2d.cu", "k_mg2d_alt.cu", "k_mg2d_alt2.cu",
                   "k_mg2d_impl.cuh")


def _code_only(text):
    """Source text without comments and blank lines (the hash follows the code, not the prose)."""
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    lines = (re.sub(r"//.*$", "", ln).rstrip() for ln in text.splitlines())
    return "\n".join(ln for ln in lines if ln)


def kernel_source_hash():
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1308_6634_gb300", "csrc")
    for f in TRAFFIC_SOURCES:
        with open(os.path.join(csrc, f), encoding="utf-8") as fh:
            h.update(_code_only(fh.read()).encode())
    return h.hexdigest()[:16]


def ncu_traffic(kclass, workload):
    """DRAM bytes per launch of a kernel class from profiles/traffic.txt, when that capture
    was taken on the current kernel sources (else None)."""
    p = os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(p):
        return None
    cur = kernel_source_hash()
    with open(p) as fh:
        for ln in fh:
            parts = ln.split()
            if len(parts) >= 4 and not ln.startswith("#") and parts[0] == kclass and parts[1] == workload \
                    and parts[3] == cur:
                return float(parts[2])
    return None


def make_inputs(W, S, seeds, torch, dev):
    """Device g for each seed: A f_true through the library's own forward map, plus noise.
    (The masked blur's mask is shared by a batch: the mask of the first seed.)"""
    gs = []
    for seed in seeds:
        f, _, z = W.inputs(seed)
        Af = S.apply_A(torch.as_tensor(f, dtype=S.dtype, device=dev))
        sig = W.noise * float(torch.linalg.vector_norm(Af.double())) / np.sqrt(Af.numel())
        g = (Af.double() + sig * torch.as_tensor(z, device=dev)).to(S.dtype).contiguous()
        gs.append(g)
    return gs


# ---- the oracle leg (cpu_baseline, accuracy, --impl reference) ------------------------------
# Everything that runs the oracle runs in spawned worker processes; the GPU side only receives
# arrays and timings from them.

_ORACLE_CACHE = {}
_BARRIER = None


def _worker_init(barrier):
    global _BARRIER
    _BARRIER = barrier


def _oracle_problem(name, seed=0):
    """(oracle operator, data g, mask) of workload `name`, seed `seed`, built once per process."""
    key = (name, seed)
    if key not in _ORACLE_CACHE:
        import oracle as O
        from paper_1308_6634_gb300 import synth
        W = synth.WORKLOADS[name]
        f, mask, z = W.inputs(seed)
        op = O.Operator(W.kind, W.shape, sigma=W.sigma, radius=W.radius, mask=mask, n_angles=W.n_angles,
                        n_bins=W.n_bins)
        _ORACLE_CACHE[key] = (op, synth.add_noise(op.A(f), W.noise, z), mask)
    return _ORACLE_CACHE[key]


def _oracle_job(task):
    """Worker: ("data", name) -> (g, mask); ("full", name, eps, k) -> a whole oracle solve of the
    data perturbed by eps (Algorithm 3, n_outer x n_inner); ("sample", name) -> seconds of one outer
    step (n_outer = 1, the workload's n_inner); ("prepare", name) builds the problem untimed."""
    import oracle as O
    from paper_1308_6634_gb300 import synth
    kind, name = task[0], task[1]
    W = synth.WORKLOADS[name]
    op, g, mask = _oracle_problem(name)
    if kind == "prepare":
        if _BARRIER is not None:
            _BARRIER.wait(timeout=600)  # one task per process
        return os.getpid()
    if kind == "data":
        return g, mask
    if kind == "full":
        eps, k = task[2], task[3]
        gp = g if eps == 0 else g * (1.0 + eps * np.random.default_rng(4242 + k).standard_normal(g.shape))
        t0 = time.perf_counter()
        r = O.solve(op, gp, W.reg, W.T, W.tau, W.n_outer, W.n_inner, W.levels, W.nu, W.cycles)
        r["seconds"] = time.perf_counter() - t0
        return r
    if kind == "sample":
        if _BARRIER is not None:
            _BARRIER.wait(timeout=600)  # all processes start together, one sample each
        t0 = time.perf_counter()
        O.solve(op, g, W.reg, W.T, W.tau, 1, W.n_inner, W.levels, W.nu, W.cycles)
        return time.perf_counter() - t0
    raise ValueError(kind)


def usable_cores():
    try:
        return len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        return os.cpu_count() or 1


def oracle_procs(requested):
    return max(1, requested if requested > 0 else min(usable_cores(), 32))


class OracleTimer:
    """P spawned oracle processes that time one outer step of workload W each, all at once: one
    such step is 1/n_outer of a solve (every outer step does the same work: the diffusivity, the
    hierarchy and coarse factorisation, and n_inner MLSQR iterations)."""

    def __init__(self, W, procs):
        import multiprocessing as mp
        self.W, self.procs = W, procs
        ctx = mp.get_context("spawn")
        self.pool = ctx.Pool(procs, initializer=_worker_init, initargs=(ctx.Barrier(procs),))
        pids = self.pool.map(_oracle_job, [("prepare", W.name)] * procs, chunksize=1)
        self.distinct = len(set(pids))

    def step(self):
        """Wall seconds of one step (P outer steps at once) and the per-process seconds."""
        t0 = time.perf_counter()
        each = self.pool.map(_oracle_job, [("sample", self.W.name)] * self.procs, chunksize=1)
        return time.perf_counter() - t0, each

    def close(self):
        self.pool.close()
        self.pool.join()


def cpu_baseline(W, procs):
    """The oracle as it stands, timed on the host cores: one outer step of the workload on one
    core, then on `procs` cores at once (independent instances)."""
    one = OracleTimer(W, 1)
    t1, _ = one.step()
    one.close()
    allc = OracleTimer(W, procs)
    tp, each = allc.step()
    allc.close()
    sample = (f"oracle (plain FP64 C, one thread per process): one whole outer step ({W.n_inner} MLSQR "
              f"iterations with the diffusivity, hierarchy and coarse factorisation) of {W.name} seed 0, i.e. "
              f"1/{W.n_outer} of a solve; every outer step does the same work")
    return {"value": procs / W.n_outer / tp, "unit": "solves/s", "cores": procs, "kind": "oracle",
            "sample": sample + f", on {procs} processes at once ({tp:.1f} s wall, slowest process "
                               f"{max(each):.1f} s)",
            "nproc": os.cpu_count(), "usable_cores": usable_cores(),
            "single_core": {"value": 1.0 / W.n_outer / t1, "unit": "solves/s", "cores": 1,
                            "outer_step_s": t1, "sample": sample + f" ({t1:.1f} s)"}}


class AccuracyLeg:
    """Whole oracle solves of the workload (seed 0), started in spawned processes before the GPU is
    touched: the unperturbed solve and two with g perturbed by one part in 1e16 (the oracle's own
    spread at this horizon).  The GPU solves the same data afterwards."""

    def __init__(self, W, n_perturbed=2):
        import multiprocessing as mp
        self.W = W
        self.pool = mp.get_context("spawn").Pool(n_perturbed + 2)
        self.data = self.pool.apply_async(_oracle_job, (("data", W.name),))
        self.full = [self.pool.apply_async(_oracle_job, (("full", W.name, 0.0, 0),))] + \
                    [self.pool.apply_async(_oracle_job, (("full", W.name, 1e-16, k),)) for k in range(n_perturbed)]

    def finish(self, gpu_runs, timeout=1800):
        """gpu_runs(g, mask) -> {label: (f, info)} of the GPU forms on the oracle's data."""
        g, mask = self.data.get(timeout=timeout)
        gpu = gpu_runs(g, mask)
        res = [r.get(timeout=timeout) for r in self.full]
        self.pool.close()
        self.pool.join()
        ref, pert = res[0], res[1:]
        relf = lambda a, b: float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))
        out = {"horizon": f"{self.W.n_outer} x {self.W.n_inner} (whole solve)",
               "oracle_seconds": ref["seconds"],
               "oracle_spread_f": [relf(r["f"], ref["f"]) for r in pert],
               "oracle_spread_R": [relf(r["R_hist"], ref["R_hist"]) for r in pert],
               "oracle_spread_resid": [relf(r["resid_hist"], ref["resid_hist"]) for r in pert]}
        for label, (f, info) in gpu.items():
            out[label] = {"f_rel_err": relf(f, ref["f"]),
                          "R_hist_rel_err": relf(info["R_hist"], ref["R_hist"]),
                          "resid_hist_rel_err": relf(info["resid_hist"], ref["resid_hist"]),
                          "rbar_first5_rel_err": relf(info["rbar_hist"][0][:5], ref["rbar_hist"][0][:5]),
                          "status": int(info["status"])}
        out["note"] = ("relative L2 errors against a whole FP64 oracle solve of the same data; the oracle's own "
                       "result moves by oracle_spread_f when g is perturbed by 1e-16 (rounding chaos of the "
                       "Krylov iteration on this ill-posed problem), so agreement below that spread is not "
                       "expected from any implementation that rounds differently; the first five residual "
                       "estimates precede the chaos")
        return out


def run_reference(args, W):
    """The oracle as the reference arm: each step is one outer step of the workload on every usable
    host core at once (independent instances), i.e. procs / n_outer solves."""
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    procs = oracle_procs(args.cpu_procs)
    timer = OracleTimer(W, procs)
    for _ in range(args.warmup):
        timer.step()
    walls, slowest = [], []
    t0 = time.perf_counter()
    for _ in range(args.steps):
        w, each = timer.step()
        walls.append(w)
        slowest.append(max(each))
    wall = time.perf_counter() - t0
    timer.close()
    step_s = float(np.mean(walls))
    value = procs / W.n_outer / step_s
    sample = (f"oracle (plain FP64 C, one thread per process): one whole outer step of {W.name} seed 0 "
              f"(1/{W.n_outer} of a solve) on each of {procs} processes at once, per step")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * step_s, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": config_of(W, 1, world, args.kappa_bf16),
        "cpu_baseline": {"value": value, "unit": "solves/s", "cores": procs, "kind": "oracle", "sample": sample,
                         "nproc": os.cpu_count(), "usable_cores": usable_cores(),
                         "distinct_processes": timer.distinct},
        "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "p50_ms": 1e3 * float(np.percentile(walls, 50)), "p99_ms": 1e3 * float(np.percentile(walls, 99)),
        "slowest_process_s": float(np.mean(slowest)), "wall_s": wall,
    }
    print(json.dumps(line), flush=True)
    return 0


def flushes_l2(W, B):
    """The GPU arm flushes L2 between timed steps when the solve's working set (about ten vectors
    per instance) is smaller than L2; otherwise the inputs are larger than L2."""
    esz = 4 if W.precision == "fp32" else 8
    return B * W_N(W) * esz * 10 < L2_BYTES


def config_of(W, B, world, kappa_bf16):
    """The workload's configuration (the same dictionary in both arms; `l2` describes the timing of
    the GPU arm)."""
    return {"workload": W.name, "shape": list(W.shape), "operator": W.kind, "n_outer": W.n_outer,
            "n_inner": W.n_inner, "reg": W.reg, "T": W.T, "tau": W.tau, "levels": W.levels, "sweeps": W.nu,
            "cycles": W.cycles, "batch": B, "parallelism": f"replicas x{world}",
            "kappa": "bf16" if kappa_bf16 else W.precision,
            "l2": "flushed between steps" if flushes_l2(W, B) else "working set larger than L2"}


def serving_stream(count, rate, budget_gb, warmup, rank, torch, dev):
    """The serving stream: Poisson arrivals of deblurring and tomography requests of mixed sizes
    served by the continuous-batching engine; solves/s = completed solves / (last completion - first
    arrival); per-request latency percentiles over `count` requests."""
    from paper_1308_6634_gb300 import serving
    reqs = serving.make_stream(count, rate=rate, seed=rank)
    data = {r.rid: serving.make_data(r, torch, dev)[0] for r in reqs}
    warm = serving.make_stream(max(8, warmup * 4), rate=1000.0, seed=10_000 + rank)
    wdata = {r.rid: serving.make_data(r, torch, dev)[0] for r in warm}
    eng = serving.Engine(hbm_budget_bytes=int(budget_gb * (1 << 30)))
    eng.run(warm, wdata, realtime=False)  # creates and warms buckets (graph capture)
    torch.cuda.synchronize()
    with ClockSampler(dev.index) as clk:
        t0 = time.perf_counter()
        eng.run(reqs, data)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
    sm = serving.summarize(reqs)
    out = {"value": sm["solves_per_s"], "unit": "solves/s", "p50_ms": sm["p50_ms"], "p99_ms": sm["p99_ms"],
           "config": {"workload": f"serve_stream_{count}_poisson{rate:g}", "sizes": list(serving.SIZES),
                      "size_p": list(serving.SIZE_P), "angles": list(serving.ANGLES), "n_outer": 10, "n_inner": 30,
                      "hbm_budget_gb": budget_gb},
           "serving": sm, "buckets": len(eng.buckets), "bucket_bytes": eng.bytes_used,
           "admission_refusals": eng.refused, "clocks": clk.summary(), "wall_s": wall,
           "warmup_requests": len(warm)}
    del eng
    torch.cuda.synchronize()
    return out


def run_serving(args):
    import torch
    rank, world, local = dist_env()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    sv = serving_stream(args.requests, args.rate, args.hbm_budget_gb, args.warmup, rank, torch, dev)
    if rank == 0:
        line = {
            "metric": "solves/s and p50/p99 ms (serving stream)", "value": sv["value"] * world,
            "unit": "solves/s", "n_gpus": world, "steps": args.requests, "warmup": sv["warmup_requests"],
            "ms_per_step": 1e3 * sv["wall_s"] / args.requests, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": dict(sv["config"], parallelism=f"replicas x{world}"),
            "p50_ms": sv["p50_ms"], "p99_ms": sv["p99_ms"], "serving": sv["serving"], "buckets": sv["buckets"],
            "bucket_bytes": sv["bucket_bytes"], "admission_refusals": sv["admission_refusals"],
            "clocks": sv["clocks"], "wall_s": sv["wall_s"],
        }
        print(json.dumps(line), flush=True)
    return 0


def roofline_of(W, B, prof, kappa_bf16=False):
    """Roofline of the dominant kernel class from an eager profile (per class: ms, launches)."""
    esz = 4 if W.precision == "fp32" else 8
    ALG_UNITS = alg_units(W, kappa_bf16)
    extra = beyond_alg_units(W)
    cand = {k: v for k, v in prof.items() if k in ALG_UNITS and v[1] > 0}
    top = max(prof.items(), key=lambda kv: kv[1][0])[0]
    total_prof = sum(v[0] for v in prof.values())
    classes_ms = {k: round(v[0], 3) for k, v in prof.items()}
    if W.kind == "joseph" and "fwd" in prof and prof["fwd"][1] > 0:
        # the projector is bound by its gathers and instruction issue, not by bytes: FP32 FMA ceiling
        ms, cnt = prof["fwd"]
        samples = joseph_samples(W.shape[0], W.n_angles, W.n_bins) * B
        achieved = 4.0 * samples / (ms / cnt / 1e3) / 1e12
        return {"bound": "alu", "kernel": "fwd", "achieved": achieved, "peak": FP32_PEAK_TFLOPS,
                "unit": "TFLOP/s", "frac": achieved / FP32_PEAK_TFLOPS,
                "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 flop x 2070 MHz",
                "traffic": None, "alg_flop_per_launch": 4.0 * samples, "samples_per_launch": samples,
                "avg_launch_us": 1e3 * ms / cnt, "launches_timed": cnt,
                "share_of_eager_device_time": ms / total_prof, "largest_class": top, "classes_ms": classes_ms}
    if not cand:
        return None
    dom = max(cand.items(), key=lambda kv: kv[1][0])[0]
    peak, src = measured_peaks()
    ms, cnt = prof[dom]
    bytes_per_launch = ALG_UNITS[dom] * esz * W_N(W) * B
    achieved = bytes_per_launch / (ms / cnt / 1e3) / 1e9
    by_class = {}
    for k2, (ms2, cnt2) in cand.items():  # every class with algorithmic bytes, same arithmetic
        a2 = ALG_UNITS[k2] * esz * W_N(W) * B / (ms2 / cnt2 / 1e3) / 1e9
        by_class[k2] = {"achieved_gbs": round(a2, 1), "frac": round(a2 / peak, 4),
                        "avg_launch_us": round(1e3 * ms2 / cnt2, 2)}
    return {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "peak_source": f"{src} (MEASURED_PEAKS.json hbm_gbs)",
            "traffic": ncu_traffic(dom, W.name), "alg_bytes_per_launch": bytes_per_launch,
            "beyond_alg_bytes_per_launch": extra.get(dom, 0.0) * esz * W_N(W) * B,
            "avg_launch_us": 1e3 * ms / cnt, "launches_timed": cnt,
            "share_of_eager_device_time": ms / total_prof, "largest_class": top,
            "classes_ms": classes_ms, "by_class": by_class}


class GpuRun:
    """One workload on the GPU: a handle with B instances, device data of B seeds, and the timing."""

    def __init__(self, W, B, torch, dev, plsqr, seeds, kappa_bf16=False, tiles=None):
        self.W, self.B, self.torch, self.dev = W, B, torch, dev
        self.S = plsqr.Solver(W.shape, W.precision, levels=W.levels, sweeps=W.nu, cycles=W.cycles, max_batch=B)
        mask = W.inputs(seeds[0])[1]
        self.S.set_operator(W.kind, sigma=W.sigma, radius=W.radius, mask=mask, n_angles=W.n_angles,
                            n_bins=W.n_bins)
        if kappa_bf16:
            self.S.set_kappa_bf16(True)
        if tiles:
            for lv, sid in enumerate(int(x) for x in tiles.split(",")):
                self.S.set_tile_shape(lv, sid)
        self.kappa_bf16 = kappa_bf16
        self.gs = make_inputs(W, self.S, seeds, torch, dev)
        self.fs = [torch.empty(W.shape, dtype=self.S.dtype, device=dev) for _ in range(B)]
        self.esz = 4 if W.precision == "fp32" else 8
        self.flush = (torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)
                      if flushes_l2(W, B) else None)

    def step(self, stats=False):
        W, B, S = self.W, self.B, self.S
        if B == 1:
            return S.solve(self.gs[0], W.reg, W.T, W.tau, W.n_outer, W.n_inner, f_out=self.fs[0], stats=stats)
        return S.solve_batch(self.gs, [W.reg] * B, [W.T] * B, [W.tau] * B, W.n_outer, W.n_inner, f_outs=self.fs,
                             stats=stats)

    def time(self, steps, warmup, world=1):
        torch = self.torch
        for _ in range(warmup):
            self.step()
        torch.cuda.synchronize()
        self.step(stats=True)
        self.launches_per_step = self.S.last_launches()
        starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
        ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
        with ClockSampler(self.dev.index) as clk:
            if world > 1:
                torch.distributed.barrier()
            torch.cuda.synchronize()
            for k in range(steps):
                if self.flush is not None:
                    self.flush.zero_()
                starts[k].record()
                self.step()
                ends[k].record()
            torch.cuda.synchronize()
            if world > 1:
                torch.distributed.barrier()
        self.per_step = np.array([s.elapsed_time(e) for s, e in zip(starts, ends)])
        self.clocks = clk.summary()
        return float(self.per_step.sum())

    def profile(self):
        self.S.profile(True)
        self.step()
        self.torch.cuda.synchronize()
        prof = self.S.profile_read()
        self.S.profile(False)
        return roofline_of(self.W, self.B, prof, self.kappa_bf16)

    def tiles(self):
        return [list(self.S.tile_shape(l)[1:]) for l in range(self.W.levels - 1) if self.S.tile_shape(l)[0] >= 0]

    def summary(self, steps):
        total_ms = float(self.per_step.sum())
        return {"value": self.B * steps / (total_ms / 1e3), "unit": "solves/s", "ms_per_step": total_ms / steps,
                "p50_ms": float(np.percentile(self.per_step, 50)), "p99_ms": float(np.percentile(self.per_step, 99)),
                "steps": steps, "gpu_launches_per_step": int(self.launches_per_step),
                "config": config_of(self.W, self.B, 1, self.kappa_bf16),
                "tiles": self.tiles(), "clocks": self.clocks}

    def close(self):
        self.S.close()
        del self.gs, self.fs, self.flush
        self.torch.cuda.synchronize()


# Other workloads measured by the default run beside the headline one: (key, workload, batch, steps,
# warm-up steps).  The batched 1024^2 forms are the throughput form of the headline workload (B
# independent instances per launch).
EXTRAS = (("deblur1024_fp32_x8", "deblur1024_fp32", 8, 2, 1),
          ("deblur1024_fp32_x32", "deblur1024_fp32", 32, 1, 1),
          ("inpaint192_fp32", "inpaint192_fp32", 1, 3, 2),
          ("tomo512_fp32", "tomo512_fp32", 1, 3, 2),
          ("tomo512_fp32_x32", "tomo512_fp32", 32, 1, 1))


def main():
    args = parse()
    if args.workload == "serve":
        return run_serving(args)
    from paper_1308_6634_gb300 import synth
    W = synth.WORKLOADS[args.workload]
    if args.impl == "reference":
        return run_reference(args, W)

    rank, world, local = dist_env()
    oracle_leg = rank == 0 and world == 1 and not args.no_cpu_baseline
    # the whole-solve oracle runs start before the GPU is touched (spawned processes)
    acc_leg = AccuracyLeg(W) if oracle_leg and not args.no_accuracy else None

    import torch
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local if world > 1 else 0)
    torch.cuda.set_device(dev)
    from paper_1308_6634_gb300 import plsqr
    B = args.batch
    run = GpuRun(W, B, torch, dev, plsqr, replica_seeds(rank, B), args.kappa_bf16, args.tiles)
    total_ms = run.time(args.steps, args.warmup, world)
    total_ms = max_over_ranks(total_ms, world, dev)
    value = world * B * args.steps / (total_ms / 1e3)
    per_step, clocks = run.per_step, run.clocks
    esz = run.esz

    # end to end through the host-buffer API: H2D of g, solve, D2H of f inside the timed region
    e2e = None
    if not args.no_e2e:
        S, gs, fs = run.S, run.gs, run.fs
        pin_g = [torch.empty(g.shape, dtype=g.dtype, pin_memory=True) for g in gs]
        for pg, g in zip(pin_g, gs):
            pg.copy_(g)
        pin_f = [torch.empty(W.shape, dtype=S.dtype, pin_memory=True) for _ in range(B)]
        e_steps = max(2, min(args.steps, 5))
        torch.cuda.synchronize()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record()
        for _ in range(e_steps):
            if B == 1:
                S.solve_host(pin_g[0].numpy(), W.reg, W.T, W.tau, W.n_outer, W.n_inner, f_out=pin_f[0].numpy())
            else:
                dg = [pg.to(dev, non_blocking=True) for pg in pin_g]
                S.solve_batch(dg, [W.reg] * B, [W.T] * B, [W.tau] * B, W.n_outer, W.n_inner, f_outs=fs, stats=False)
                for pf, f in zip(pin_f, fs):
                    pf.copy_(f, non_blocking=True)
                torch.cuda.synchronize()
        t1.record()
        torch.cuda.synchronize()
        e_ms = t0.elapsed_time(t1)
        e2e = {"value": world * B * e_steps / (e_ms / 1e3), "unit": "solves/s",
               "h2d_bytes_per_step": int(B * gs[0].numel() * esz), "d2h_bytes_per_step": int(B * W_N(W) * esz)}

    # roofline of the dominant kernel class: eager profiling pass, CUDA events on the launch stream
    roofline = None if args.no_profile else run.profile()

    # the plain form beside it: the same workload with the same kernels instantiated in double,
    # one instance per call, no CUDA graph
    fp64_single, S64 = None, None
    if rank == 0 and world == 1 and not args.no_fp64_single and W.precision == "fp32":
        fp64_single, S64 = time_fp64_single(W, plsqr, torch, dev, run.gs[0])

    # the other workloads (single GPU only: the headline's timed work stays the one multi-GPU job)
    workloads = None
    if rank == 0 and world == 1 and not args.no_extras and W.name == "deblur1024_fp32":
        workloads = {}
        for key, wname, b, st, wu in EXTRAS:
            r2 = GpuRun(synth.WORKLOADS[wname], b, torch, dev, plsqr, replica_seeds(0, b))
            r2.time(st, wu)
            workloads[key] = dict(r2.summary(st), roofline=r2.profile())
            r2.close()
        workloads["serve_2000_poisson200"] = serving_stream(2000, 200.0, args.hbm_budget_gb, 3, 0, torch, dev)
        # the same mix at an arrival rate inside the engine's capacity: latency without a growing queue
        workloads["serve_800_poisson40"] = serving_stream(800, 40.0, args.hbm_budget_gb, 3, 0, torch, dev)

    accuracy = None
    if acc_leg is not None:
        def gpu_runs(g, mask):
            out = {}
            gd = torch.as_tensor(g, dtype=run.S.dtype, device=dev)
            f, info = run.S.solve(gd, W.reg, W.T, W.tau, W.n_outer, W.n_inner)
            out["gpu"] = (f.double().cpu().numpy(), info)
            if S64 is not None:
                f64, info64 = S64.solve(torch.as_tensor(g, dtype=torch.float64, device=dev), W.reg, W.T, W.tau,
                                        W.n_outer, W.n_inner)
                out["gpu_fp64_single"] = (f64.cpu().numpy(), info64)
            return out
        accuracy = acc_leg.finish(gpu_runs)

    cpu = cpu_baseline(W, oracle_procs(args.cpu_procs)) if oracle_leg else None

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32" if W.precision == "fp32" else "f64",
            "data": "synthetic",
            "config": config_of(W, B, world, args.kappa_bf16),
            "tiles": run.tiles(),
            "p50_ms": float(np.percentile(per_step, 50)), "p99_ms": float(np.percentile(per_step, 99)),
            "gpu_launches": int(run.launches_per_step * args.steps),
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks, "accuracy": accuracy,
            "fp64_single": fp64_single, "workloads": workloads,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def W_N(W):
    return int(np.prod(W.shape))


def replica_seeds(rank, B):
    """Seeds of the B instances a rank solves: replicas of the workload, disjoint across ranks."""
    return [rank * B + b for b in range(B)]


def max_over_ranks(x, world, device):
    """The largest value of x over the ranks of the default process group (the timing rule)."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def time_fp64_single(W, plsqr, torch, dev, g32, steps=2):
    """solves/s of the double-precision single-instance form without graph replay, and the
    relative difference of its reconstruction from the single-precision one on the same data."""
    os.environ["PLSQR_GRAPH"] = "0"
    try:
        S = plsqr.Solver(W.shape, "fp64", levels=W.levels, sweeps=W.nu, cycles=W.cycles)
    finally:
        os.environ.pop("PLSQR_GRAPH", None)
    S.set_operator(W.kind, sigma=W.sigma, radius=W.radius, mask=W.inputs(0)[1], n_angles=W.n_angles,
                   n_bins=W.n_bins)
    g = g32.double()
    f = torch.empty(W.shape, dtype=torch.float64, device=dev)
    S.solve(g, W.reg, W.T, W.tau, W.n_outer, W.n_inner, f_out=f)  # warm-up
    torch.cuda.synchronize()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record()
    for _ in range(steps):
        S.solve(g, W.reg, W.T, W.tau, W.n_outer, W.n_inner, f_out=f)
    t1.record()
    torch.cuda.synchronize()
    ms = t0.elapsed_time(t1) / steps
    S32 = plsqr.Solver(W.shape, "fp32", levels=W.levels, sweeps=W.nu, cycles=W.cycles)
    S32.set_operator(W.kind, sigma=W.sigma, radius=W.radius, mask=W.inputs(0)[1], n_angles=W.n_angles,
                     n_bins=W.n_bins)
    f32, _ = S32.solve(g32, W.reg, W.T, W.tau, W.n_outer, W.n_inner)
    diff = float(torch.linalg.vector_norm(f32.double() - f) / torch.linalg.vector_norm(f))
    S32.close()
    return {"value": 1e3 / ms, "unit": "solves/s", "ms_per_solve": ms, "batch": 1, "graph": False,
            "dtype": "f64", "steps": steps, "rel_diff_fp32_vs_fp64_f": diff}, S


if __name__ == "__main__":
    sys.exit(main())
