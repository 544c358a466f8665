"""Run full FMM evaluations of a named synthetic workload on cuda:0.

    python -m paper_0809_1810_gb300.run_workload --workload uniform_1m --steps 3 [--p P --L L]

Each step is one complete fmm2d_velocity call (tree build to velocities);
this is the command the profiler summaries under profiles/ are taken with.
Prints the mean step time from CUDA events.
"""
from __future__ import annotations

import argparse
import os
import sys

import numpy as np
import torch

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import workloads as W  # noqa: E402

from . import Plan  # noqa: E402

WORKLOADS = {
    "lamb_oseen_4096": lambda: W.lamb_oseen_lattice(64, p=10, L=3, dtype=np.float32),
    "uniform_1m": W.uniform_1m,
    "uniform_4m": lambda: W.uniform_random(1 << 22, 2, 2.0 / 2048, sigma_over_h=2.0, p=16, L=8),
    "uniform_16m": lambda: W.uniform_random(1 << 24, 2, 2.0 / 4096, sigma_over_h=2.0, p=16,
                                            L=9),
    "clustered_16m": W.clustered_16m,
}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="uniform_1m", choices=sorted(WORKLOADS))
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp32_tc", "fp64"])
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=2)
    ap.add_argument("--p", type=int, default=None, help="override the workload's p")
    ap.add_argument("--L", type=int, default=None, help="override the workload's L")
    ap.add_argument("--cutoff", type=float, default=0.0,
                    help="cutoff a of Sec. 4.1 in units of sigma (0: the plain 3x3 rule)")
    ap.add_argument("--phases", action="store_true",
                    help="also print the mean per-phase times (events inside the graph)")
    args = ap.parse_args()
    w = WORKLOADS[args.workload]()
    if args.p is not None:
        w.p = args.p
    if args.L is not None:
        w.L = args.L
    dt = torch.float64 if args.precision == "fp64" else torch.float32
    xy = torch.tensor(np.stack([w.x, w.y], 1), dtype=dt, device="cuda")
    g = torch.tensor(w.gamma, dtype=dt, device="cuda")
    uv = torch.empty((w.n, 2), dtype=dt, device="cuda")
    with Plan(w.p, w.L, w.sigma, args.precision, root=w.root, max_n=w.n,
              cutoff=args.cutoff * w.sigma) as plan:
        if args.phases:
            plan.set_timing(max(args.steps, 1))
        for _ in range(args.warmup):
            plan.velocity(xy, g, out=uv)
        plan.check()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(args.steps):
            plan.velocity(xy, g, out=uv)
        b.record()
        plan.check()
        print(f"{args.workload} {args.precision}: n={w.n} p={w.p} L={w.L} a={args.cutoff}sigma "
              f"{a.elapsed_time(b) / max(args.steps, 1):.4f} ms/step, "
              f"{plan.kernels_per_call()} kernels/step")
        if args.phases:
            ph = [plan.phase_ms(a) for a in range(max(args.steps, 1))]
            print("  phases (ms): " + ", ".join(
                f"{k} {np.mean([q[k] for q in ph]):.4f}" for k in ph[0]))


if __name__ == "__main__":
    main()
