"""Train the correction network on solver-generated pairs and compare
learned 64^3, plain 64^3 and plain 128^3 runs against the 256^3 run
restricted to 64^3 (error and GPU time).  Prints a markdown report and,
with --json, writes the numbers.

    python -m paper_1004_1680_gb300.learned_experiment [--train-seeds 10]
        [--steps-per-seed 200] [--epochs 6] [--eval-seeds 4] [--eval-steps 200]

Turbulence as in the 512^3 workload (k^-2 for 2 <= k <= 8, Mach 1, beta 1),
with the optional pressure floor 1e-3 in every run (the long 256^3 runs leave
the floor-free scheme's positivity range otherwise).  Training seeds are
0.., held-out seeds 10000..; pairs are every coarse step of each training
trajectory.
"""
from __future__ import annotations

import argparse
import json
import sys
import time

import numpy as np
import torch

from . import learned, mhd


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--train-seeds", type=int, default=10)
    ap.add_argument("--steps-per-seed", type=int, default=200)
    ap.add_argument("--epochs", type=int, default=6)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--eval-seeds", type=int, default=4)
    ap.add_argument("--eval-steps", type=int, default=200)
    ap.add_argument("--alphas", default="1.0",
                    help="comma-separated scales of the applied correction to evaluate (1.0: as trained)")
    ap.add_argument("--json", default=None)
    args = ap.parse_args(argv)
    log = lambda s: print(s, file=sys.stderr, flush=True)  # noqa: E731

    t0 = time.perf_counter()
    inputs, targets = learned.generate_pairs(range(args.train_seeds), args.steps_per_seed)
    torch.cuda.synchronize()
    log(f"pairs: {inputs.shape[0]} in {time.perf_counter() - t0:.1f} s")
    norm = learned.make_norm(inputs, targets, inputs.shape[-1])
    t1 = time.perf_counter()
    net, hist = learned.train(inputs, targets, norm, args.epochs, lr=args.lr, log=log)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t1
    assert mhd.conv_error() == 0
    del inputs, targets
    torch.cuda.empty_cache()
    alphas = [float(a) for a in args.alphas.split(",")]
    per_alpha = {}
    for alpha in alphas:
        corr = learned.Corrector(net, norm, (64, 64, 64), alpha=alpha)
        res = []
        for k in range(args.eval_seeds):
            errs, gpu_ms, T, nclip = learned.evaluate(corr, 10000 + k, nsteps=args.eval_steps)
            res.append((errs, gpu_ms, T, nclip))
            log(f"alpha {alpha} seed {10000 + k}: T={T:.3f} " +
                " ".join(f"{n}={errs[n].mean():.4f}" for n in errs) + f" clip={nclip}")
        per_alpha[alpha] = res
    res = per_alpha[alphas[0]]
    runs = ["plain64", "learned64", "plain128"]
    mean_err = {r: float(np.mean([x[0][r].mean() for x in res])) for r in runs}
    final_err = {r: float(np.mean([x[0][r][-1].mean() for x in res])) for r in runs}
    per_field = {r: np.mean([x[0][r].mean(axis=0) for x in res], axis=0).tolist() for r in runs}
    curve = {r: np.mean([x[0][r].mean(axis=1) for x in res], axis=0).tolist() for r in runs}
    gpu = {r: float(np.mean([x[1][r] for x in res])) for r in runs + ["ref"]}
    out = {"train_pairs": args.train_seeds * args.steps_per_seed, "epochs": args.epochs, "train_s": train_s,
           "loss_history": hist, "eval_seeds": args.eval_seeds, "eval_steps": args.eval_steps,
           "mean_nrmse": mean_err, "final_nrmse": final_err, "per_field_nrmse": per_field,
           "nrmse_every_20_steps": curve,
           "gpu_ms_per_run": gpu, "clipped_cells": [x[3] for x in res],
           "alphas": {str(a): {"mean_nrmse": float(np.mean([x[0]["learned64"].mean() for x in r])),
                               "final_nrmse": float(np.mean([x[0]["learned64"][-1].mean() for x in r])),
                               "nrmse_every_20_steps": np.mean([x[0]["learned64"].mean(axis=1) for x in r],
                                                               axis=0).tolist()}
                      for a, r in per_alpha.items()},
           "claim_lower_error_than_plain128": mean_err["learned64"] < mean_err["plain128"],
           "claim_less_gpu_time_than_plain128": gpu["learned64"] < gpu["plain128"]}
    print("| run | mean NRMSE (8 fields, every 20 steps) | NRMSE at the last step | GPU ms per run |")
    print("|---|---|---|---|")
    for r in runs:
        print(f"| {r} | {mean_err[r]:.4f} | {final_err[r]:.4f} | {gpu[r]:.1f} |")
    print(f"| 256^3 reference | - | - | {gpu['ref']:.1f} |")
    print()
    print("per-field mean NRMSE (rho, m_x, m_y, m_z, e, b_x, b_y, b_z):")
    for r in runs:
        print(f"  {r}: " + ", ".join(f"{v:.4f}" for v in per_field[r]))
    print()
    print("mean NRMSE after 20, 40, ... coarse steps:")
    for r in runs:
        print(f"  {r}: " + ", ".join(f"{v:.4f}" for v in curve[r]))
    if len(alphas) > 1:
        print()
        print("learned 64^3 with the correction scaled by alpha (mean NRMSE; after 20, 40, ... steps):")
        for a, r in out["alphas"].items():
            print(f"  alpha {a}: {r['mean_nrmse']:.4f}; " + ", ".join(f"{v:.3f}" for v in r["nrmse_every_20_steps"]))
    print(f"training: {out['train_pairs']} pairs x {args.epochs} epochs in {train_s:.1f} s; "
          f"loss history {[round(h, 4) for h in hist]}")
    print(f"claim (learned 64^3 error < plain 128^3): {out['claim_lower_error_than_plain128']}; "
          f"(learned 64^3 GPU time < plain 128^3): {out['claim_less_gpu_time_than_plain128']}")
    if args.json:
        with open(args.json, "w") as f:
            json.dump(out, f, indent=1)
    return 0


if __name__ == "__main__":
    sys.exit(main())
