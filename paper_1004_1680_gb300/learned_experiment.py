"""Train the correction network on solver-generated pairs and compare
learned 64^3, plain 64^3 and plain 128^3 runs against the 256^3 run
restricted to 64^3 (error and GPU time).  Prints a markdown report and,
with --json, writes the numbers.

    python -m paper_1004_1680_gb300.learned_experiment [--train-seeds 2000]
        [--pairs-per-seed 1] [--t-max 200] [--epochs 6] [--val-seeds 8]
        [--eval-seeds 64] [--eval-steps 200]

Turbulence as in the 512^3 workload (k^-2 for 2 <= k <= 8, Mach 1, beta 1),
with the optional pressure floor 1e-3 in every run (the long 256^3 runs leave
the floor-free scheme's positivity range otherwise).  Training seeds 0..,
each giving pairs at coarse step counts drawn from [0, t_max); the scale
of the applied correction is chosen on validation seeds 20000..; held-out
seeds 10000.. are used for the comparison only.
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
    ap.add_argument("--train-seeds", type=int, default=2000)
    ap.add_argument("--pairs-per-seed", type=int, default=1)
    ap.add_argument("--t-max", type=int, default=200, help="pairs at coarse step counts drawn from [0, t_max)")
    ap.add_argument("--rollout", type=int, default=1)
    ap.add_argument("--epochs", type=int, default=6)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--val-seeds", type=int, default=8)
    ap.add_argument("--eval-seeds", type=int, default=64)
    ap.add_argument("--eval-steps", type=int, default=200)
    ap.add_argument("--alphas", default="0,0.25,0.5,0.75,1.0",
                    help="comma-separated scales of the applied correction tried on the validation seeds")
    ap.add_argument("--json", default=None)
    args = ap.parse_args(argv)
    log = lambda s: print(s, file=sys.stderr, flush=True)  # noqa: E731

    t0 = time.perf_counter()
    inputs, targets = learned.generate_pairs(range(args.train_seeds), steps_per_seed=args.pairs_per_seed,
                                             t_max=args.t_max, rollout=args.rollout, log=log)
    torch.cuda.synchronize()
    pairs_s = time.perf_counter() - t0
    log(f"pairs: {inputs.shape[0]} in {pairs_s:.1f} s")
    norm = learned.make_norm(inputs, targets, inputs.shape[-1])
    t1 = time.perf_counter()
    net, hist = learned.train(inputs, targets, norm, args.epochs, lr=args.lr, log=log)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t1
    assert mhd.conv_error() == 0
    npairs = int(inputs.shape[0])
    del inputs, targets
    torch.cuda.empty_cache()
    alphas = [float(a) for a in args.alphas.split(",")]
    best, val_means = learned.choose_alpha(net, norm, [20000 + k for k in range(args.val_seeds)], alphas=alphas,
                                           nsteps=args.eval_steps, log=log)
    log(f"alpha chosen on validation seeds: {best} ({val_means})")
    corrs = [learned.Corrector(net, norm, (64, 64, 64), alpha=a) for a in (best, 1.0)]
    res = []
    left_out = []
    for k in range(args.eval_seeds):
        r = learned.evaluate_safe(corrs, 10000 + k, log=log, nsteps=args.eval_steps)
        if r is None:
            left_out.append(10000 + k)
            continue
        errs, gpu_ms, T, nclip = r
        errs["learned64"] = errs.pop("learned64/0")
        errs["learned64_alpha1"] = errs.pop("learned64/1")
        gpu_ms["learned64"] = gpu_ms.pop("learned64/0")
        gpu_ms["learned64_alpha1"] = gpu_ms.pop("learned64/1")
        res.append((errs, gpu_ms, T, nclip))
        log(f"seed {10000 + k}: T={T:.3f} " + " ".join(f"{n}={errs[n].mean():.4f}" for n in errs))
    runs = ["plain64", "learned64", "learned64_alpha1", "plain128"]
    mean_err = {r: float(np.mean([x[0][r].mean() for x in res])) for r in runs}
    final_err = {r: float(np.mean([x[0][r][-1].mean() for x in res])) for r in runs}
    per_field = {r: np.mean([x[0][r].mean(axis=0) for x in res], axis=0).tolist() for r in runs}
    curve = {r: np.mean([x[0][r].mean(axis=1) for x in res], axis=0).tolist() for r in runs}
    gpu = {r: float(np.mean([x[1][r] for x in res])) for r in runs + ["ref"]}
    wins = int(sum(x[0]["learned64"].mean() < x[0]["plain64"].mean() for x in res))
    out = {"train_seeds": args.train_seeds, "train_pairs": npairs, "pairs_per_seed": args.pairs_per_seed,
           "t_max": args.t_max, "epochs": args.epochs, "pairs_s": pairs_s, "train_s": train_s,
           "loss_history": hist, "val_seeds": args.val_seeds, "validation_mean_nrmse": val_means,
           "alpha": best, "eval_seeds": args.eval_seeds, "eval_steps": args.eval_steps,
           "mean_nrmse": mean_err, "final_nrmse": final_err, "per_field_nrmse": per_field,
           "nrmse_every_20_steps": curve, "gpu_ms_per_run": gpu, "clipped_cells": [x[3] for x in res],
           "seeds_where_learned_beats_plain64": wins, "eval_seeds_used": len(res),
           "eval_seeds_left_out": left_out, "train_seeds_skipped": getattr(learned.generate_pairs, "skipped", []),
           "claim_lower_error_than_plain64": mean_err["learned64"] < mean_err["plain64"],
           "claim_lower_error_than_plain128": mean_err["learned64"] < mean_err["plain128"],
           "claim_less_gpu_time_than_plain128": gpu["learned64"] < gpu["plain128"]}
    print(f"alpha (chosen on validation seeds 20000..{20000 + args.val_seeds - 1}): {best}; "
          f"validation mean NRMSE by alpha: {val_means}")
    print("| run | mean NRMSE (8 fields, every 20 steps) | NRMSE at the last step | GPU ms per run |")
    print("|---|---|---|---|")
    for r in runs:
        print(f"| {r} | {mean_err[r]:.4f} | {final_err[r]:.4f} | {gpu[r]:.1f} |")
    print(f"| 256^3 reference | - | - | {gpu['ref']:.1f} |")
    print()
    print(f"held-out seeds where learned 64^3 beats plain 64^3: {wins} of {len(res)} "
          f"(left out, a run left the valid states: {left_out}); training seeds skipped: "
          f"{out['train_seeds_skipped']}")
    print("per-field mean NRMSE (rho, m_x, m_y, m_z, e, b_x, b_y, b_z):")
    for r in runs:
        print(f"  {r}: " + ", ".join(f"{v:.4f}" for v in per_field[r]))
    print()
    print("mean NRMSE after 20, 40, ... coarse steps:")
    for r in runs:
        print(f"  {r}: " + ", ".join(f"{v:.4f}" for v in curve[r]))
    print(f"training: {npairs} pairs from {args.train_seeds} seeds ({pairs_s:.0f} s) x {args.epochs} epochs in "
          f"{train_s:.1f} s; loss history {[round(h, 4) for h in hist]}")
    print(f"claims: learned 64^3 error < plain 64^3: {out['claim_lower_error_than_plain64']}; "
          f"< plain 128^3: {out['claim_lower_error_than_plain128']}; "
          f"GPU time < plain 128^3: {out['claim_less_gpu_time_than_plain128']}")
    if args.json:
        with open(args.json, "w") as f:
            json.dump(out, f, indent=1)
    return 0


if __name__ == "__main__":
    sys.exit(main())
