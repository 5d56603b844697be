"""Timing of the FP64 CPU oracle (test infrastructure): cell-updates per
second of full steps (CFL + 12 sweeps) on the turbulence recipe, with one
thread and with all host threads, printed as a markdown table.

    python tests/oracle_timing.py [--sizes 32,64,128] [--steps 5] [--big 256]
"""
from __future__ import annotations

import argparse
import os
import platform
import time

import sys

import torch

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import oracle  # noqa: E402
from paper_1004_1680_gb300 import initial_conditions as ic  # noqa: E402

G = 5.0 / 3.0


def rate(n: int, steps: int, threads: int) -> float:
    s = ic.turbulence((n, n, n), seed=0, dtype=torch.float64).numpy().copy()
    oracle.set_threads(threads)
    oracle.step(s, oracle.cfl_dt(s, G, 0.7), G)          # warm-up
    t0 = time.perf_counter()
    for _ in range(steps):
        oracle.step(s, oracle.cfl_dt(s, G, 0.7), G)
    return n ** 3 * steps / (time.perf_counter() - t0)


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--sizes", default="32,64,128")
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--big", type=int, default=256, help="edge of a box timed for one step, all threads (0: skip)")
    args = ap.parse_args(argv)
    oracle.build()
    allt = os.cpu_count() or 1
    print(f"FP64 oracle on {platform.machine()}, {allt} hardware threads ({platform.processor() or 'cpu'}); "
          f"cell-updates/s of full steps on the turbulence recipe\n")
    print("| box | steps | 1 thread | all threads | speed-up |")
    print("|---|---|---|---|---|")
    for n in (int(x) for x in args.sizes.split(",")):
        r1 = rate(n, args.steps, 1)
        ra = rate(n, args.steps, allt)
        print(f"| {n}^3 | {args.steps} | {r1 / 1e6:.2f} M | {ra / 1e6:.2f} M | {ra / r1:.1f} |", flush=True)
    if args.big:
        ra = rate(args.big, 1, allt)
        print(f"| {args.big}^3 | 1 | - | {ra / 1e6:.2f} M | - |", flush=True)
    oracle.set_threads(allt)
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
