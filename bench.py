"""Benchmark: solves/s of the priorconditioned lagged-diffusivity solver on one workload.

One step = one batch of B complete solves (Algorithm 3: n_outer lagged-diffusivity steps,
each with n_inner MLSQR iterations and a fresh V-cycle priorconditioner) of the 1024x1024
FP32 deblurring workload (Gaussian blur sigma 4 truncated at radius 12, 1% noise,
Perona-Malik log regulariser T = 5e-2, tau = 1e-3, 15 x 50 iterations, 6-level V-cycle with
2 red-black sweeps per side), inputs resident in device memory.  Multi-GPU runs are replicas
(independent instances per rank, no collective on the data path; weak scaling).

JSON line keys beyond the base contract: p50_ms/p99_ms (per-step latency), roofline of the
dominant kernel class (eager profiling pass with CUDA events on the launch stream),
cpu_baseline (the FP64 CPU oracle on a bounded sample, extrapolated), e2e (host buffers, copies
inside the timed region), clocks (nvidia-smi sampled during the timed region), accuracy (the
first MLSQR residual estimates against the oracle's).

--impl reference times the FP64 CPU oracle itself on the same workload and metric.
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
    instances).  2D V-cycle (finest level, mean of the pre- and post-smoothing launches):
    pre reads b, kappa and the reciprocal diagonal and writes x and the restricted residual (1/4);
    post reads x_in, b, kappa, the reciprocal diagonal and the coarse correction (1/4) and writes x.
    kappa in bfloat16 counts half."""
    n = W.n_inner
    two_d_blur = W.kind in ("blur", "blur_mask") and len(W.shape) == 2
    fused_update = two_d_blur and W.precision == "fp32" and W.radius[0] == W.radius[1] and W.radius[0] in (6, 9, 12, 15)
    fwd = (3.0 + 7.0 * (n - 1)) / n if fused_update else 3.0
    if len(W.shape) == 2:
        k = 0.5 if kappa_bf16 else 1.0
        return {"fwd": fwd, "adj": 3.0, "gs_fine": ((3.25 + k) + (4.25 + k)) / 2}
    # 3D: one launch per red-black half sweep: x of the other colour (1/2), kappa (1),
    # b of this colour (1/2) in, x of this colour (1/2) out
    return {"fwd": fwd, "adj": 3.0, "gs_fine": 2.5}


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


def cpu_baseline(W, budget_s=20.0):
    """The FP64 CPU oracle on a bounded sample: one outer step with i1 and i2 inner
    iterations; the difference gives the cost of one iteration, the rest the per-outer-step
    cost (diffusivity, hierarchy, coarse factorisation, initialisation); both extrapolated
    to the full n_outer x n_inner solve."""
    import oracle as O
    from paper_1308_6634_gb300 import synth
    f, mask, z = W.inputs(0)
    op = O.Operator(W.kind, W.shape, sigma=W.sigma, radius=W.radius, mask=mask, n_angles=W.n_angles,
                    n_bins=W.n_bins)
    g = synth.add_noise(op.A(f), W.noise, z)
    i1, i2 = 2, 6
    t0 = time.perf_counter()
    r1 = O.solve(op, g, W.reg, W.T, W.tau, 1, i1, W.levels, W.nu, W.cycles)
    t1 = time.perf_counter()
    r2 = O.solve(op, g, W.reg, W.T, W.tau, 1, i2, W.levels, W.nu, W.cycles)
    t2 = time.perf_counter()
    per_iter = max((t2 - t1) - (t1 - t0), 1e-9) / (i2 - i1)
    per_outer = max((t1 - t0) - i1 * per_iter, 0.0)
    t_solve = W.n_outer * (per_outer + W.n_inner * per_iter)
    return dict(value=1.0 / t_solve, t_solve=t_solve, per_iter=per_iter, per_outer=per_outer,
                sample_s=t2 - t0, rbar=r2["rbar_hist"][0], g=g, mask=mask, i2=i2,
                sample=f"oracle: 1 outer step x {i1} and x {i2} inner iterations on seed 0 ({t2 - t0:.1f} s), "
                f"extrapolated to {W.n_outer} x {W.n_inner}")


def run_reference(args, W):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    for _ in range(args.warmup):
        pass  # the oracle has no warm-up state
    vals = []
    t0 = time.perf_counter()
    info = None
    for _ in range(args.steps):
        info = cpu_baseline(W)
        vals.append(info["t_solve"])
    wall = time.perf_counter() - t0
    t_solve = float(np.mean(vals))
    line = {
        "impl": "reference", "metric": METRIC, "value": 1.0 / t_solve, "unit": "solves/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_solve, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": W.name, "shape": list(W.shape), "n_outer": W.n_outer, "n_inner": W.n_inner,
                   "batch": 1, "parallelism": "replicas"},
        "cpu_baseline": {"value": 1.0 / t_solve, "unit": "solves/s", "cores": 1, "kind": "oracle",
                         "sample": info["sample"]},
        "e2e": {"value": 1.0 / t_solve, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "wall_s": wall,
    }
    print(json.dumps(line), flush=True)
    return 0


def run_serving(args):
    """The serving stream: Poisson arrivals of deblurring and tomography requests of mixed sizes
    served by the continuous-batching engine; value = completed solves / (last completion - first
    arrival); per-request latency percentiles over --requests requests."""
    import torch
    from paper_1308_6634_gb300 import serving
    rank, world, local = dist_env()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    count = args.requests
    reqs = serving.make_stream(count, rate=args.rate, seed=rank)
    data = {r.rid: serving.make_data(r, torch, dev)[0] for r in reqs}
    warm = serving.make_stream(max(8, args.warmup * 4), rate=1000.0, seed=10_000 + rank)
    wdata = {r.rid: serving.make_data(r, torch, dev)[0] for r in warm}
    eng = serving.Engine(hbm_budget_bytes=int(args.hbm_budget_gb * (1 << 30)))
    eng.run(warm, wdata, realtime=False)  # creates and warms buckets (graph capture)
    torch.cuda.synchronize()
    with ClockSampler(dev.index) as clk:
        t0 = time.perf_counter()
        eng.run(reqs, data)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
    sm = serving.summarize(reqs)
    if rank == 0:
        line = {
            "metric": "solves/s and p50/p99 ms (serving stream)", "value": sm["solves_per_s"] * world,
            "unit": "solves/s", "n_gpus": world, "steps": count, "warmup": len(warm),
            "ms_per_step": 1e3 * wall / count, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"serve_stream_{count}_poisson{args.rate:g}", "sizes": list(serving.SIZES),
                       "size_p": list(serving.SIZE_P), "angles": list(serving.ANGLES), "n_outer": 10,
                       "n_inner": 30, "parallelism": f"replicas x{world}", "hbm_budget_gb": args.hbm_budget_gb},
            "p50_ms": sm["p50_ms"], "p99_ms": sm["p99_ms"], "serving": sm,
            "buckets": len(eng.buckets), "bucket_bytes": eng.bytes_used, "admission_refusals": eng.refused,
            "clocks": clk.summary(), "wall_s": wall,
        }
        print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse()
    if args.workload == "serve":
        return run_serving(args)
    from paper_1308_6634_gb300 import synth
    W = synth.WORKLOADS[args.workload]
    if args.impl == "reference":
        return run_reference(args, W)

    import torch
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local if world > 1 else 0)
    torch.cuda.set_device(dev)
    from paper_1308_6634_gb300 import plsqr
    B = args.batch
    S = plsqr.Solver(W.shape, W.precision, levels=W.levels, sweeps=W.nu, cycles=W.cycles, max_batch=B)
    seeds = replica_seeds(rank, B)
    mask = W.inputs(seeds[0])[1]
    S.set_operator(W.kind, sigma=W.sigma, radius=W.radius, mask=mask, n_angles=W.n_angles, n_bins=W.n_bins)
    if args.kappa_bf16:
        S.set_kappa_bf16(True)
    if args.tiles:
        for lv, sid in enumerate(int(x) for x in args.tiles.split(",")):
            S.set_tile_shape(lv, sid)
    gs = make_inputs(W, S, seeds, torch, dev)
    fs = [torch.empty(W.shape, dtype=S.dtype, device=dev) for _ in range(B)]
    regs, Ts, taus = [W.reg] * B, [W.T] * B, [W.tau] * B

    def step(stats=False):
        if B == 1:
            return S.solve(gs[0], W.reg, W.T, W.tau, W.n_outer, W.n_inner, f_out=fs[0], stats=stats)
        return S.solve_batch(gs, regs, Ts, taus, W.n_outer, W.n_inner, f_outs=fs, stats=stats)

    esz = 4 if W.precision == "fp32" else 8
    working_set = B * int(np.prod(W.shape)) * esz * 10
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev) if working_set < L2_BYTES else None

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    _, info = step(stats=True)
    launches_per_step = S.last_launches()

    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    with ClockSampler(dev.index) as clk:
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        for k in range(args.steps):
            if flush is not None:
                flush.zero_()
            starts[k].record()
            step()
            ends[k].record()
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
    per_step = np.array([s.elapsed_time(e) for s, e in zip(starts, ends)])
    total_ms = float(per_step.sum())
    total_ms = max_over_ranks(total_ms, world, dev)
    value = world * B * args.steps / (total_ms / 1e3)

    # end to end through the host-buffer API: H2D of g, solve, D2H of f inside the timed region
    e2e = None
    if not args.no_e2e:
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
                S.solve_batch(dg, regs, Ts, taus, W.n_outer, W.n_inner, f_outs=fs, stats=False)
                for pf, f in zip(pin_f, fs):
                    pf.copy_(f, non_blocking=True)
                torch.cuda.synchronize()
        t1.record()
        torch.cuda.synchronize()
        e_ms = t0.elapsed_time(t1)
        e2e = {"value": world * B * e_steps / (e_ms / 1e3), "unit": "solves/s",
               "h2d_bytes_per_step": int(B * gs[0].numel() * esz), "d2h_bytes_per_step": int(B * W_N(W) * esz)}

    # roofline of the dominant kernel class: eager profiling pass, CUDA events on the launch stream
    roofline = None
    if not args.no_profile:
        S.profile(True)
        step()
        torch.cuda.synchronize()
        prof = S.profile_read()
        S.profile(False)
        ALG_UNITS = alg_units(W, args.kappa_bf16)
        cand = {k: v for k, v in prof.items() if k in ALG_UNITS and v[1] > 0}
        top = max(prof.items(), key=lambda kv: kv[1][0])[0]
        dom = max(cand.items(), key=lambda kv: kv[1][0])[0] if cand else None
        peak, src = measured_peaks()
        if W.kind == "joseph" and "fwd" in prof and prof["fwd"][1] > 0:
            # the projector is bound by its gathers and instruction issue, not by bytes: FP32 FMA ceiling
            ms, cnt = prof["fwd"]
            samples = joseph_samples(W.shape[0], W.n_angles, W.n_bins) * B
            achieved = 4.0 * samples / (ms / cnt / 1e3) / 1e12
            total_prof = sum(v[0] for v in prof.values())
            roofline = {"bound": "alu", "kernel": "fwd", "achieved": achieved, "peak": FP32_PEAK_TFLOPS,
                        "unit": "TFLOP/s", "frac": achieved / FP32_PEAK_TFLOPS,
                        "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 flop x 2070 MHz",
                        "traffic": None, "alg_flop_per_launch": 4.0 * samples, "samples_per_launch": samples,
                        "avg_launch_us": 1e3 * ms / cnt, "launches_timed": cnt,
                        "share_of_eager_device_time": ms / total_prof, "largest_class": top,
                        "classes_ms": {k: round(v[0], 3) for k, v in prof.items()}}
            dom = None
        if dom is not None:
            ms, cnt = prof[dom]
            bytes_per_launch = ALG_UNITS[dom] * esz * W_N(W) * B
            achieved = bytes_per_launch / (ms / cnt / 1e3) / 1e9
            total_prof = sum(v[0] for v in prof.values())
            by_class = {}
            for k2, (ms2, cnt2) in cand.items():  # every class with algorithmic bytes, same arithmetic
                a2 = ALG_UNITS[k2] * esz * W_N(W) * B / (ms2 / cnt2 / 1e3) / 1e9
                by_class[k2] = {"achieved_gbs": round(a2, 1), "frac": round(a2 / peak, 4),
                                "avg_launch_us": round(1e3 * ms2 / cnt2, 2)}
            roofline = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
                        "frac": achieved / peak, "peak_source": f"{src} (MEASURED_PEAKS.json hbm_gbs)",
                        "traffic": ncu_traffic(dom, W.name), "alg_bytes_per_launch": bytes_per_launch,
                        "avg_launch_us": 1e3 * ms / cnt, "launches_timed": cnt,
                        "share_of_eager_device_time": ms / total_prof, "largest_class": top,
                        "classes_ms": {k: round(v[0], 3) for k, v in prof.items()}, "by_class": by_class}

    # the plain form beside it: the same workload with the same kernels instantiated in double,
    # one instance per call, no CUDA graph
    fp64_single = None
    if rank == 0 and world == 1 and not args.no_fp64_single and W.precision == "fp32":
        fp64_single = time_fp64_single(W, plsqr, torch, dev, gs[0])

    cpu = None
    acc = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cb = cpu_baseline(W)
        cpu = {"value": cb["value"], "unit": "solves/s", "cores": 1, "kind": "oracle", "sample": cb["sample"]}
        # accuracy on the oracle's own data g: the same first outer step on the GPU
        ref = cb["rbar"]
        S1 = plsqr.Solver(W.shape, W.precision, levels=W.levels, sweeps=W.nu, cycles=W.cycles)
        S1.set_operator(W.kind, sigma=W.sigma, radius=W.radius, mask=cb["mask"], n_angles=W.n_angles,
                        n_bins=W.n_bins)
        if args.kappa_bf16:
            S1.set_kappa_bf16(True)
        _, inf1 = S1.solve(torch.as_tensor(cb["g"], dtype=S1.dtype, device=dev), W.reg, W.T, W.tau, 1, cb["i2"])
        got = inf1["rbar_hist"][0]
        acc = {"rbar_rel_err_first4": float(np.linalg.norm(got[:4] - ref[:4]) / np.linalg.norm(ref[:4])),
               "rbar_rel_err_per_iter": [float(abs(a - b) / abs(b)) for a, b in zip(got, ref)],
               "note": "||rbar_i|| of the first outer step on the oracle's data against the oracle's; rounding "
                       "chaos sets in after a few iterations (tomography: from the fifth), so later entries "
                       "measure the problem's sensitivity; long-horizon parity is tested against the oracle's "
                       "rounding envelope (tests/)"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32" if W.precision == "fp32" else "f64",
            "data": "synthetic",
            "config": {"workload": W.name, "shape": list(W.shape), "operator": W.kind, "n_outer": W.n_outer,
                       "n_inner": W.n_inner, "reg": W.reg, "T": W.T, "tau": W.tau, "levels": W.levels,
                       "sweeps": W.nu, "cycles": W.cycles, "batch": B, "parallelism": f"replicas x{world}",
                       "kappa": "bf16" if args.kappa_bf16 else W.precision,
                       "tiles": [list(S.tile_shape(l)[1:]) for l in range(W.levels - 1) if S.tile_shape(l)[0] >= 0],
                       "l2": "flushed between steps" if flush is not None else "working set larger than L2"},
            "p50_ms": float(np.percentile(per_step, 50)), "p99_ms": float(np.percentile(per_step, 99)),
            "gpu_launches": int(launches_per_step * args.steps),
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "clocks": clk.summary(), "accuracy": acc,
            "fp64_single": fp64_single,
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
    return {"value": 1e3 / ms, "unit": "solves/s", "ms_per_solve": ms, "batch": 1, "graph": False,
            "dtype": "f64", "steps": steps, "rel_diff_fp32_vs_fp64_f": diff}


if __name__ == "__main__":
    sys.exit(main())
