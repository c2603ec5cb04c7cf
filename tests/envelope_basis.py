"""Measured basis of the rounding envelopes in envelope.py (test infrastructure; CPU only).

For each long-horizon parity case this runs the reference computation of envelope.py (the
oracle for double-precision handles, the float32 model for single-precision ones) K times on
perturbed data g (1 + eps xi_k), eps cycling through a set of magnitudes, and reports

  * the spread of each output (f, the ||rbar|| history, R(f^k), ||g - A f^k||) against the
    unperturbed oracle: minimum / median / maximum over the K runs, per magnitude;
  * the ratio of a fresh draw to the maximum of m others (the envelope a test computes from m
    perturbed runs), by resampling the K runs: its 99th and 99.9th percentiles, and the largest
    ratio seen.

A double-precision GPU result behaves like a fresh draw when its rounding differs from the
oracle's and nothing else does, so the 99.9th percentile of that ratio is the factor the envelope
needs to keep a correct implementation from failing more often than once in a thousand runs.  Nothing here is an expected
value: the script only sizes tolerances.

    python tests/envelope_basis.py [--cases a,b] [--runs K] [--procs P]
"""
import argparse
import multiprocessing as mp
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))
sys.path.insert(0, HERE)

KEYS = ("f", "rbar_hist", "R_hist", "resid_hist")
EPS_FP64 = (1e-16, 1e-15, 1e-14)


def _cases():
    from test_gpu_parity import SOLVE_CASES
    return SOLVE_CASES


def _task(args):
    from envelope import solve_task
    name, kind, eps, k = args
    W, n_outer, n_inner = _cases()[name]
    r = solve_task((kind, W, n_outer, n_inner, eps, k))
    return {key: np.asarray(r[key]) for key in KEYS if key in r}


def _err(a, b):
    from envelope import rel
    return rel(a, b)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--cases", default=None)
    ap.add_argument("--runs", type=int, default=30)
    ap.add_argument("--procs", type=int, default=os.cpu_count() or 1)
    ap.add_argument("--others", default="9,29", help="envelope sizes (perturbed runs) to evaluate")
    a = ap.parse_args()
    a.others = [int(v) for v in a.others.split(",")]
    from envelope import EPS
    cases = a.cases.split(",") if a.cases else sorted(_cases())
    rng = np.random.default_rng(0)
    ctx = mp.get_context("spawn")
    with ctx.Pool(a.procs) as pool:
        for name in cases:
            t0 = time.time()
            W = _cases()[name][0]
            kind = "oracle" if W.precision == "fp64" else "model32"
            eps = EPS_FP64 if W.precision == "fp64" else EPS["fp32"]
            base = _task((name, "oracle", 0.0, 0))
            tasks = [(name, kind, eps[k % len(eps)], k) for k in range(a.runs)]
            res = pool.map(_task, tasks)
            print(f"{name} ({W.precision}, {kind}, {a.runs} runs, eps {', '.join(f'{e:g}' for e in eps)})")
            for key in KEYS:
                if key not in base or key not in res[0]:
                    continue
                b = base[key][1:] if key == "R_hist" else base[key]  # R(f^0) = 0 exactly
                x = np.array([_err(r[key][1:] if key == "R_hist" else r[key], b) for r in res])
                per = " | ".join(
                    f"{e:g}: {np.min(x[i::len(eps)]):.1e}/{np.median(x[i::len(eps)]):.1e}/{np.max(x[i::len(eps)]):.1e}"
                    for i, e in enumerate(eps))
                print(f"  {key:10s} spread min/median/max  {per}")
                for m in a.others:
                    if m + 1 > len(x):
                        continue
                    ratios = []
                    for _ in range(20000):
                        idx = rng.choice(len(x), m + 1, replace=False)
                        ratios.append(x[idx[0]] / max(x[idx[1:]].max(), 1e-300))
                    ratios = np.array(ratios)
                    print(f"  {key:10s} fresh draw / max of {m}: p99 {np.quantile(ratios, 0.99):.2f}, "
                          f"p99.9 {np.quantile(ratios, 0.999):.2f}, largest {ratios.max():.2f}")
            print(f"  ({time.time() - t0:.0f} s)", flush=True)


if __name__ == "__main__":
    main()
