"""Precision statement: per-field error of the FP32 GPU path against the FP64
oracle on the workloads of the hot path (run on a GPU machine; prints a
markdown table).

    python tests/precision_report.py [--full] [--json profiles/precision.json]

Errors per field f (rho, m_x, m_y, m_z, e, b_x, b_y, b_z):
  max   = max |gpu - oracle| / max(max|oracle_f|, S_f)     (S_f: background scale)
  L2    = ||gpu - oracle||_2 / max(||oracle_f||_2, S_f sqrt(N))
Both paths start from the same FP32-rounded state and take the same dt.
--json also writes the table as a record keyed by the hash of the sweep
sources, which bench.py attaches to its JSON line while the kernels are
unchanged.
"""
import argparse
import json
import math
import os
import sys

import numpy as np
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1004_1680_gb300 import initial_conditions as ic  # noqa: E402
from paper_1004_1680_gb300 import mhd  # noqa: E402
from tests.parity_util import G, field_scales, sub_block  # noqa: E402

FIELDS = ["rho", "m_x", "m_y", "m_z", "e", "b_x", "b_y", "b_z"]


def errors(g, o, S):
    mx, l2 = [], []
    n = o[0].size
    for q in range(8):
        d = g[q].astype(np.float64) - o[q]
        den = max(float(np.max(np.abs(o[q]))), S[q]) or 1.0
        mx.append(float(np.max(np.abs(d))) / den)
        den2 = max(float(np.sqrt(np.sum(o[q] ** 2))), S[q] * math.sqrt(n)) or 1.0
        l2.append(float(np.sqrt(np.sum(d ** 2))) / den2)
    return mx, l2


def run_pair(st64, nsteps, cfl=0.7):
    s = ic.as_oracle_input(st64)
    S = field_scales(s)
    nz, ny, nx = s.shape[1:]
    box = mhd.Box(nx, ny, nz, gamma=G)
    box.set_state(st64.to(torch.float32).contiguous().cuda())
    for _ in range(nsteps):
        dt = oracle.cfl_dt(s, G, cfl)
        oracle.step(s, dt, G)
        box.step(dt)
    g = box.get_state().cpu().numpy()
    box.close()
    return errors(g, s, S)


def run_sampled(n=512, L=24, H=24):
    torch.cuda.empty_cache()
    box = mhd.Box(n, n, n, gamma=G)      # the library's memory first, as bench.py does
    st = ic.turbulence((n, n, n), seed=0, device="cuda", dtype=torch.float32)
    box.set_state(st)
    init = st.cpu().numpy()
    del st
    torch.cuda.empty_cache()
    dt = box.cfl_dt(0.7)
    box.step(dt)
    out = box.get_state().cpu().numpy()
    box.close()
    rng = np.random.default_rng(0)
    gs, os_ = [], []
    for lo in [(0, 0, 0)] + [tuple(rng.integers(0, n, 3)) for _ in range(3)]:
        nb = L + 2 * H
        blk = sub_block(init, [c - H for c in lo], [nb] * 3).astype(np.float64)
        oracle.step(blk, dt * n / nb, G)
        os_.append(blk[:, H:H + L, H:H + L, H:H + L])
        gs.append(sub_block(out, lo, [L] * 3))
    o = np.concatenate([x.reshape(8, -1) for x in os_], axis=1)
    g = np.concatenate([x.reshape(8, -1) for x in gs], axis=1)
    return errors(g, o, field_scales(sub_block(init, (0, 0, 0), (64, 64, 64)).astype(np.float64)))


def run_ensemble_members(nsteps=4, cfl=0.7):
    """Members of the 256-box ensemble recipe (per-axis sizes in
    {32,48,64,96}, rng 2024; box b seeded 1000 + b with its own Mach and
    beta), the first 16 boxes advanced together in one ensemble with the
    pressure floor of the ensemble workload; 4 of them (0, 5, 10, 15) against
    the oracle with the same floor and each box's own CFL dt."""
    specs = ic.ensemble_specs(256, seed=2024)[:16]
    dims = [sp["dims"] for sp in specs]
    ens = mhd.Ensemble(dims, gamma=G)
    ens.set_pressure_floor(1e-3)
    sts = []
    for b, sp in enumerate(specs):
        st = ic.turbulence(sp["dims"], seed=sp["seed"], mach=sp["mach"], beta=sp["beta"], dtype=torch.float64)
        sts.append(st)
        ens.set_state(b, st.to(torch.float32).contiguous().cuda())
    ens.run(nsteps, cfl)
    gs, os_, scales = [], [], []
    oracle.set_pressure_floor(1e-3)
    try:
        for b in (0, 5, 10, 15):
            s = ic.as_oracle_input(sts[b])
            scales.append(field_scales(s))
            for _ in range(nsteps):
                oracle.step(s, oracle.cfl_dt(s, G, cfl), G)
            os_.append(s.reshape(8, -1))
            gs.append(ens.get_state(b).cpu().numpy().reshape(8, -1))
    finally:
        oracle.set_pressure_floor(0.0)
    ens.close()
    S = [max(sc[q] for sc in scales) for q in range(8)]
    return errors(np.concatenate(gs, axis=1), np.concatenate(os_, axis=1), S)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--full", action="store_true", help="include 256^3, 512^3 and 1024^3 cases")
    ap.add_argument("--json", default="", help="also write the table to this JSON file")
    args = ap.parse_args()
    cases = []
    alf, _ = ic.alfven_wave((32, 32, 32), k_int=(1, 1, 1), amp=1e-6)
    cases.append(("Alfven 32^3 amp 1e-6, 1 step", lambda: run_pair(alf, 1)))
    cases.append(("Alfven 32^3 amp 1e-6, 20 steps", lambda: run_pair(alf, 20)))
    sod = ic.sod((32, 32, 32))
    cases.append(("shock tube 32^3, 1 step", lambda: run_pair(sod, 1)))
    cases.append(("shock tube 32^3, 20 steps", lambda: run_pair(sod, 20)))
    turb = ic.turbulence((64, 64, 64), seed=0, dtype=torch.float64)
    cases.append(("turbulence 64^3 (k 2..8), 1 step", lambda: run_pair(turb, 1)))
    cases.append(("turbulence 64^3 (k 2..8), 10 steps", lambda: run_pair(turb, 10)))
    cases.append(("ensemble members (4 of 16 boxes, 32..96 per axis, p_floor 1e-3), 4 steps",
                  run_ensemble_members))
    if args.full:
        ot = ic.orszag_tang((256, 256, 256))
        cases.append(("Orszag-Tang 256^3, 1 step", lambda: run_pair(ot, 1)))
        cases.append(("turbulence 512^3, 1 step (4 sampled 24^3 blocks)", run_sampled))
        cases.append(("turbulence 1024^3, 1 step (4 sampled 24^3 blocks)", lambda: run_sampled(1024)))
    print("| case | error | " + " | ".join(FIELDS) + " |")
    print("|---|---|" + "---|" * 8)
    rec = {"fields": FIELDS, "cases": {}}
    for name, fn in cases:
        mx, l2 = fn()
        rec["cases"][name] = {"max": mx, "l2": l2}
        print(f"| {name} | max | " + " | ".join(f"{v:.1e}" for v in mx) + " |")
        print(f"| | L2 | " + " | ".join(f"{v:.1e}" for v in l2) + " |")
        sys.stdout.flush()
    if args.json:
        from bench import kernel_source_hash
        rec["source_hash"] = kernel_source_hash()
        rec["command"] = "python tests/precision_report.py" + (" --full" if args.full else "") + \
            f" --json {args.json}"
        rec["worst_max"] = [max(c["max"][q] for c in rec["cases"].values()) for q in range(8)]
        with open(args.json, "w") as f:
            json.dump(rec, f, indent=1)


if __name__ == "__main__":
    main()
