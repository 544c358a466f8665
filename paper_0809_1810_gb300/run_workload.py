"""Run full FMM evaluations of a named synthetic workload on cuda:0.

    python -m paper_0809_1810_gb300.run_workload --workload uniform_1m --steps 3 [--p P --L L]
    python -m paper_0809_1810_gb300.run_workload --workload batch_sweep --steps 3 [--per-leaf 0 32]

Each step is one complete fmm2d_velocity call (tree build to velocities),
or for batch_sweep one fmm2d_batch_velocity call over the 512 instances of
the batched benchmark (FP32_TC, each instance with the Sec. 4.1 cutoff for
1e-6 where its leaves are narrower than it, default launch shapes); this is
the command the profiler summaries under profiles/ are taken with.  Prints
the mean step time from CUDA events.
"""
from __future__ import annotations

import argparse
import os
import sys

import numpy as np
import torch

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import workloads as W  # noqa: E402

from . import BatchPlan, Plan, cutoff_for  # noqa: E402

WORKLOADS = {
    "lamb_oseen_4096": lambda: W.lamb_oseen_lattice(64, p=10, L=3, dtype=np.float32),
    "uniform_1m": W.uniform_1m,
    "uniform_4m": lambda: W.uniform_random(1 << 22, 2, 2.0 / 2048, sigma_over_h=2.0, p=16, L=8),
    "uniform_16m": lambda: W.uniform_random(1 << 24, 2, 2.0 / 4096, sigma_over_h=2.0, p=16,
                                            L=9),
    "clustered_16m": W.clustered_16m,
}


def run_batch_sweep(args):
    ws = [W.make_instance(s) for s in W.batch_instances(512, seed=3)[:args.instances]]
    if args.per_leaf:  # one class of mean leaf occupancy, as its own batch
        lo, hi = args.per_leaf
        ws = [w for w in ws if lo <= w.n / 4 ** w.L < hi]
    xy = torch.tensor(np.concatenate([np.stack([w.x, w.y], 1) for w in ws]), device="cuda")
    g = torch.tensor(np.concatenate([w.gamma for w in ws]), device="cuda")
    insts = [{"n": w.n, "p": w.p, "L": w.L, "sigma": w.sigma, "root": w.root,
              "cutoff": cutoff_for(w.sigma, w.root[2] / 2 ** w.L, 1e-6) if w.L >= 2 else 0.0}
             for w in ws]
    with BatchPlan(insts, precision="fp32_tc") as bp:
        uv = torch.empty((bp.n_total, 2), dtype=torch.float32, device="cuda")
        for _ in range(args.warmup):
            bp.velocity(xy, g, out=uv)
        bp.check()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(args.steps):
            bp.velocity(xy, g, out=uv)
        b.record()
        bp.check()
        print(f"batch_sweep fp32_tc: {len(ws)} instances, n={bp.n_total} "
              f"{a.elapsed_time(b) / max(args.steps, 1):.4f} ms/batch")
        if args.phases:
            ph = bp.profile(xy, g, uv)
            print("  phases (ms): " + ", ".join(f"{k} {v:.4f}" for k, v in ph.items()))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="uniform_1m",
                    choices=sorted(WORKLOADS) + ["batch_sweep"])
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp32_tc", "fp64"])
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=2)
    ap.add_argument("--p", type=int, default=None, help="override the workload's p")
    ap.add_argument("--L", type=int, default=None, help="override the workload's L")
    ap.add_argument("--cutoff", type=float, default=0.0,
                    help="cutoff a of Sec. 4.1 in units of sigma (0: the plain 3x3 rule)")
    ap.add_argument("--phases", action="store_true",
                    help="also print the mean per-phase times (events inside the graph)")
    ap.add_argument("--instances", type=int, default=512,
                    help="batch_sweep: the first this many of its 512 instances")
    ap.add_argument("--per-leaf", type=float, nargs=2, default=None, metavar=("LO", "HI"),
                    help="batch_sweep: only the instances with LO <= n / 4^L < HI")
    args = ap.parse_args()
    if args.workload == "batch_sweep":
        run_batch_sweep(args)
        return
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
