#!/usr/bin/env python3
"""Throughput of the dimensionally split MHD grid update on GB300.

Metric: cell-updates/s per full step (one step = CFL timestep + fluid/magnetic
sweeps x, y, z then z, y, x), on 512^3 periodic decaying MHD turbulence
(rho = 1, p = 1, k^-2 spectrum for 2 <= k <= 8, rms Mach 1, beta 1, seed 0),
FP32 state.  The state (4.3 GB) is far larger than L2, so no flush is needed
between steps.

Prints one JSON line (rank 0).  `value` is device time (CUDA events on the
library's stream) with the state resident in HBM; `e2e` is the same metric
through the C ABI with host buffers, the host->device copy of the state and
the device->host copy of the result inside every timed step (with
`e2e.link_bound`, the rate the measured host link allows); `roofline` is
the dominant kernel's algorithmic bytes over its measured launch time;
`cpu_baseline` times the FP64 oracle on the host cores on a bounded sample.

--impl reference times the FP64 CPU oracle instead (no installable reference
implementation exists for this paper).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "cell-updates/s per full step"
UNIT = "cell-updates/s"
# Algorithmic bytes per cell of one launch (each field read once, written once):
#   fluid sweep: reads rho, m (3), e, b (3) = 32 B, writes rho, m, e = 20 B
#   magnetic sweep: reads rho, m_d, b (3) = 20 B, writes b (3) = 12 B
ALGO_BYTES = {"fluid": 52, "mag": 32}
TRANSPOSE_BYTES = 64   # x<->y exchange: read and write 8 fields
DIAG_BYTES = 32        # FP64 diagnostics: read 8 fields
STEP_BYTES = 384  # 6 sweeps x (read + write of 8 FP32 fields): the full-step model
P_FLOOR_ENSEMBLE = 1e-3


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=50)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--size", type=int, default=512)
    p.add_argument("--cfl", type=float, default=0.7)
    p.add_argument("--seed", type=int, default=0)
    p.add_argument("--e2e-steps", type=int, default=20)
    p.add_argument("--diag-reps", type=int, default=10,
                   help="FP64 diagnostics passes timed on the final state (0: skip)")
    p.add_argument("--cpu-sample", type=int, default=128, help="edge of the oracle's sample box")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--ensemble-steps", type=int, default=100,
                   help="steps of the 256-box ensemble measurement (0: skip)")
    p.add_argument("--limiter", choices=["vanleer", "minmod", "superbee"], default="vanleer",
                   help="slope limiter (van Leer is the paper's; the others are ablations)")
    p.add_argument("--xpath", type=int, choices=[0, 1, 2, 3], default=0,
                   help="x sweep path (0 automatic; 3 = every axis through transposes, the paper's data flow)")
    p.add_argument("--seg", type=int, default=0,
                   help="pencil segment length for every axis (0: the library's choice)")
    p.add_argument("--freezing", choices=["bound", "fast", "pencil"], default="bound",
                   help="freezing speed (the bound is the paper-reading default; fast is an ablation)")
    p.add_argument("--shard", action="store_true",
                   help="one box of --size^3 cut into z-slabs over the ranks (strong scaling; the default "
                        "for several GPUs is one box per rank, weak scaling)")
    p.add_argument("--fp64", action="store_true",
                   help="time the FP64 path (mhd_create_f64, an ablation) instead of the FP32 one")
    p.add_argument("--fusion", type=int, choices=[0, 1], default=1,
                   help="1: the two middle z magnetic sweeps of a step as one launch (bitwise the same state)")
    p.add_argument("--tma", type=int, choices=[0, 1], default=1,
                   help="1: the y and z kernel-axis fluid sweeps stage their input with TMA tile copies "
                        "(bitwise the same state)")
    p.add_argument("--bc", default="",
                   help="non-periodic axes, e.g. x=outflow,z=reflecting (4 ghost cells at each end "
                        "inside the box; the paper's runs are periodic)")
    p.add_argument("--mach", type=float, default=1.0, help="rms Mach number of the turbulence recipe")
    p.add_argument("--beta", type=float, default=1.0, help="plasma beta of the turbulence recipe")
    p.add_argument("--learned-reps", type=int, default=20,
                   help="timed applications of the 64^3 learned correction (0: skip)")
    return p.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# --------------------------------------------------------------------------
# clocks during the timed region

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_uuid: str | None):
        self.uuid = device_uuid
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                   "-lms", "50"]
            if self.uuid:
                cmd += ["-i", self.uuid]
            self.proc = subprocess.Popen(cmd, stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self) -> dict | None:
        if self.proc is None:
            return None
        time.sleep(0.1)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) == 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# --------------------------------------------------------------------------
# CPU baseline: the FP64 oracle, as it stands, on a bounded sample

def cpu_baseline(n: int, seed: int, cfl: float, budget_s: float = 15.0, min_steps: int = 1):
    import numpy as np
    import torch

    import oracle
    from paper_1004_1680_gb300 import initial_conditions as ic
    s = ic.turbulence((n, n, n), seed=seed, dtype=torch.float64).numpy().copy()
    g = 5.0 / 3.0
    steps = 0
    t0 = time.perf_counter()
    while steps < min_steps or time.perf_counter() - t0 < budget_s:
        oracle.step(s, oracle.cfl_dt(s, g, cfl), g)
        steps += 1
        if steps >= 50:
            break
    el = time.perf_counter() - t0
    return {"value": n ** 3 * steps / el, "unit": UNIT, "cores": oracle.threads(), "kind": "oracle",
            "sample": f"{n}^3 box of the same turbulence recipe (seed {seed}), {steps} full steps "
                      f"(CFL dt each), FP64, {el:.1f} s"}


# --------------------------------------------------------------------------

def kernel_source_hash() -> str:
    h = hashlib.sha256()
    for name in ("sweep_fluid.cuh", "sweep_mag.cuh", "sweep_row.cuh", "mhd_device.cuh", "tma.cuh"):
        with open(os.path.join(ROOT, "paper_1004_1680_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def measured_traffic(kernel: str, n: int):
    """DRAM bytes per launch from a committed ncu capture, if it was taken on
    the current kernel source (else None)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            rec = json.load(f)
    except (OSError, ValueError):
        return None
    r = rec.get(kernel)
    if not r or r.get("source_hash") != kernel_source_hash():
        return None
    return r["bytes_per_cell"] * n ** 3


def measured_issue(kernel: str):
    """Warp instructions per cell of a kernel family from the committed ncu
    capture (smsp__inst_executed.sum over cells), if it was taken on the
    current kernel source (else None)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            rec = json.load(f)
    except (OSError, ValueError):
        return None
    r = rec.get(kernel)
    if not r or r.get("source_hash") != kernel_source_hash():
        return None
    return r.get("warp_instructions_per_cell")


def precision_record():
    """Per-field error of the FP32 path against the FP64 oracle
    (tests/precision_report.py --full --json), if it was taken on the current
    kernel source (else None): the worst max error of every field over all
    cases, and the 512^3 sampled case in full."""
    path = os.path.join(ROOT, "profiles", "precision.json")
    try:
        with open(path) as f:
            rec = json.load(f)
    except (OSError, ValueError):
        return None
    if rec.get("source_hash") != kernel_source_hash():
        return None
    cases = rec.get("cases", {})
    big = {k: v for k, v in cases.items() if k.startswith("turbulence 512^3")}
    return {"fields": rec["fields"], "worst_max_over_cases": rec.get("worst_max"),
            "cases": len(cases), "turbulence_512": next(iter(big.values()), None),
            "source": "profiles/precision.json", "command": rec.get("command")}


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except (OSError, ValueError, KeyError):
        return 6800.0, "fallback"


def bf16_peak():
    """Dense BF16 tensor peak (TFLOP/s) for a kernel timed alone: measured burst, else fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["bf16_tflops"]), "measured bf16 burst"
    except (OSError, ValueError, KeyError):
        return 1900.0, "fallback bf16 burst"


def ensemble_leg(args, world=1):
    """256 independent periodic boxes, per-axis sizes drawn from {32,48,64,96}
    (rng 2024), box b seeded 1000+b with its own rms Mach and beta; one batched
    launch per sweep, per-box CFL dt, the run replayed as one CUDA graph."""
    import torch

    from paper_1004_1680_gb300 import initial_conditions as ic
    from paper_1004_1680_gb300 import mhd
    specs = ic.ensemble_specs(256, seed=2024)
    dims = [sp["dims"] for sp in specs]
    ens = mhd.Ensemble(dims, gamma=5.0 / 3.0)
    # The strongly magnetised (beta down to 0.3) supersonic boxes of this recipe
    # reach p <= 0 within 100 steps with the floor-free scheme; the optional
    # pressure floor keeps every box valid (it adds at most ~1.5% energy).
    ens.set_pressure_floor(P_FLOOR_ENSEMBLE)
    for b, sp in enumerate(specs):
        st = ic.turbulence(sp["dims"], seed=sp["seed"], mach=sp["mach"], beta=sp["beta"],
                           device="cuda", dtype=torch.float32)
        ens.set_state(b, st)
    torch.cuda.synchronize()
    cells = sum(a * b * c for a, b, c in dims)
    xp, sd = ens.autotune(args.cfl)
    ens.run(args.ensemble_steps, args.cfl)      # capture + warm-up of the timed graph
    invalid_warm = int(np.sum(ens.cfl_dt_safe(args.cfl) == 0.0))
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    e0.record(ens.stream)
    ens.run(args.ensemble_steps, args.cfl)
    e1.record(ens.stream)
    torch.cuda.synchronize()
    secs = max_over_ranks([e0.elapsed_time(e1) / 1e3], world)[0]
    invalid = int(np.sum(ens.cfl_dt_safe(args.cfl) == 0.0))
    peak, peak_kind = peaks()
    gbs = STEP_BYTES * cells * args.ensemble_steps / secs / 1e9
    out = {"value": whole_job_rate(cells * args.ensemble_steps, world, secs), "unit": UNIT, "boxes": len(dims),
           "roofline": {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s", "frac": gbs / peak,
                        "model_bytes_per_cell": STEP_BYTES, "peak_kind": peak_kind,
                        "note": "full-step model (6 sweeps x read + write of 8 fields) over all boxes; "
                                f"state {2 * 32 * cells / 1e9:.1f} GB in two copies > L2"},
           "cells": cells, "steps": args.ensemble_steps, "ms_per_step": 1e3 * secs / args.ensemble_steps,
           "tuning": {"xpath": xp, "segdiv": sd}, "pressure_floor": P_FLOOR_ENSEMBLE,
           "invalid_boxes": invalid,
           "invalid_boxes_after_warmup": invalid_warm,
           "launch": "one CUDA graph per run; 1 launch per sweep for all boxes"}
    ens.close()
    return out


def learned_leg(args):
    """Kernels of the learned coarse-grid correction on a 64^3 box: each
    tensor-core convolution layer (forward, 2 * 27 * cin * cout flop per cell),
    and one whole correction (normalise, 4 layers, projection, clipped
    correction).  Weights are a random initialisation of the architecture;
    the activations (<= 16.8 MB) are L2-resident, so the layers are timed
    back to back."""
    import torch

    from paper_1004_1680_gb300 import initial_conditions as ic
    from paper_1004_1680_gb300 import learned, mhd
    n = (64, 64, 64)
    cells = n[0] * n[1] * n[2]
    st = ic.turbulence(n, seed=args.seed, device="cuda", dtype=torch.float32)
    net = learned.CorrectionNet(seed=0)
    norm = learned.Norm(mu=[float(st[q].mean()) for q in range(8)],
                        inv_sigma=[1.0 / max(float(st[q].std()), 1e-3) for q in range(8)],
                        out_scale=[1e-3] * 5 + [1e-5], loss_weight=[1.0] * 8)
    corr = learned.Corrector(net, norm, n)
    mhd.cnn_normalize(st, norm.mu, norm.inv_sigma, out=corr.x)
    stream = torch.cuda.current_stream()

    def graph_ms(fn):
        """Device time of one fn(): `reps` calls captured in a CUDA graph (so
        host launch overhead is not timed), replayed after a warm-up replay."""
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            for _ in range(args.learned_reps):
                fn()
        g.replay()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        g.replay()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / args.learned_reps

    layer_ms, layer_flop = [], []
    h = corr.x
    for li, (ci, co) in enumerate(learned.LAYERS):
        last = li == len(learned.LAYERS) - 1
        out = mhd.conv3d(h, net.img[li], n, ci, co, bias=net.b[li], relu=not last,
                         out_bf16=not last, out_f32=last)
        yb, yf = out
        run = lambda: mhd.conv3d_into(h, net.img[li], n, ci, co, yb, yf, bias=net.b[li],  # noqa: E731
                                      relu=not last)
        layer_ms.append(graph_ms(run))
        layer_flop.append(2.0 * 27 * ci * co * cells)
        h = yf if last else yb
    work = st.clone()
    correction_ms = graph_ms(lambda: corr.apply(work, corr.predict(st)))
    # weight gradient of a 32 -> 32 layer (CUDA cores; FP32 atomics accumulate)
    acts_in = mhd.conv3d(corr.x, net.img[0], n, 8, 32, bias=net.b[0], relu=True)[0]
    gy = (torch.randn(cells, 32, device="cuda") * 0.1).to(torch.bfloat16)
    gw = torch.zeros(32 * 32 * 27, device="cuda")
    gb = torch.zeros(32, device="cuda")
    wgrad_ms = graph_ms(lambda: mhd.conv3d_wgrad(acts_in, gy, n, 32, 32, gw, gb))
    if mhd.conv_error():
        raise RuntimeError("a tensor-core wait gave up")
    peak, peak_kind = bf16_peak()
    tf = sum(layer_flop) / (sum(layer_ms) / 1e3) / 1e12
    out = {"grid": "64^3", "layers": [f"{ci}->{co}" for ci, co in learned.LAYERS],
           "layer_ms": layer_ms,
           "layer_tflops": [f / (t / 1e3) / 1e12 for f, t in zip(layer_flop, layer_ms)],
           "conv_flop_per_application": sum(layer_flop),
           "roofline": {"bound": "tensor", "achieved": tf, "peak": peak, "unit": "TFLOP/s",
                        "frac": tf / peak, "kernel": "conv3d (tcgen05 implicit GEMM)",
                        "peak_kind": peak_kind},
           "correction_ms": correction_ms,
           "wgrad_32x32_ms": wgrad_ms,
           "wgrad_32x32_tflops": 2.0 * 27 * 32 * 32 * cells / (wgrad_ms / 1e3) / 1e12,
           "timing": "CUDA graph of the repeated calls (device time only)",
           "reps": args.learned_reps}
    return out


def max_over_ranks(values, world, device="cuda"):
    """Each rank's timings -> the maximum over ranks of each (the slowest
    rank sets the whole job's time); identity for a single rank."""
    if world <= 1:
        return [float(v) for v in values]
    import torch
    t = torch.tensor([float(v) for v in values], device=device, dtype=torch.float64)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return [float(v) for v in t.tolist()]


def host_link_rate(host, out_host, reps=2):
    """GB/s each way of pinned host <-> HBM copies running in both directions
    at once (the regime of the pipelined end-to-end leg): each of the 8 fields
    in, and one field's worth out, per field, on two streams."""
    import torch

    d_in = torch.empty_like(host[0], device="cuda")
    d_out = torch.zeros_like(d_in)
    sa, sb = torch.cuda.Stream(), torch.cuda.Stream()
    best = math.inf
    for _ in range(reps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for q in range(host.shape[0]):
            with torch.cuda.stream(sa):
                d_in.copy_(host[q], non_blocking=True)
            with torch.cuda.stream(sb):
                out_host[q].copy_(d_out, non_blocking=True)
        torch.cuda.synchronize()
        best = min(best, time.perf_counter() - t0)
    del d_in, d_out
    return host.numel() * host.element_size() / best / 1e9


def whole_job_rate(units_per_rank, world, secs):
    """Units processed by all ranks together (replicas: each rank the same
    amount) over the slowest rank's time."""
    return units_per_rank * world / secs


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    import torch

    import oracle
    from paper_1004_1680_gb300 import initial_conditions as ic
    n = args.cpu_sample
    g = 5.0 / 3.0
    s = ic.turbulence((n, n, n), seed=args.seed, dtype=torch.float64).numpy().copy()
    for _ in range(args.warmup):
        oracle.step(s, oracle.cfl_dt(s, g, args.cfl), g)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.step(s, oracle.cfl_dt(s, g, args.cfl), g)
    el = time.perf_counter() - t0
    value = n ** 3 * args.steps / el
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "impl": "reference",
           "config": {"workload": f"decaying MHD turbulence {args.size}^3, periodic", "n": args.size,
                      "seed": args.seed, "cfl": args.cfl,
                      "sample": f"each step timed on a {n}^3 box of the same recipe (FP64 CPU oracle)"},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.threads(), "kind": "oracle",
                            "sample": f"{n}^3 turbulence, {args.steps} timed full steps"},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)
    return 0


def run_ours(args, rank, world, local):
    import torch

    from paper_1004_1680_gb300 import initial_conditions as ic
    from paper_1004_1680_gb300 import mhd

    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    n = args.size
    N = n ** 3
    box = mhd.Box(n, n, n, gamma=5.0 / 3.0)
    box.set_scheme(args.limiter, args.freezing)
    if args.xpath:
        box.set_xpath(args.xpath)
    box.set_fusion(bool(args.fusion))
    box.set_tma(bool(args.tma))
    if args.seg:
        box.set_segments(args.seg, args.seg, args.seg)
    bcs = {}
    for item in filter(None, args.bc.split(",")):
        axis, mode = item.split("=")
        box.set_boundary("xyz".index(axis), mode)
        bcs[axis] = mode
    stream = torch.cuda.current_stream()
    st = ic.turbulence((n, n, n), seed=args.seed + rank, mach=args.mach, beta=args.beta, device="cuda",
                       dtype=torch.float32)
    host = st.cpu().pin_memory()     # for the end-to-end leg
    box.set_state(st)
    torch.cuda.synchronize()
    del st
    torch.cuda.empty_cache()

    box.run(args.warmup, args.cfl)
    box.cfl_dt(args.cfl)               # raises if the state went invalid
    start = box.get_state()            # the traced pass below repeats the same steps
    # 12 sweeps, step control, up to 6 transposes (x path 3); with ghost
    # layers a fill per non-periodic axis before every sweep; with the
    # per-pencil freezing speed a reduction pass before every fluid sweep
    launches_per_step = 19 + 12 * len(bcs) + (6 if args.freezing == "pencil" else 0)  # + speed passes

    uuid = None
    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(local).uuid)
    except Exception:
        uuid = None
    clocks = ClockSampler(uuid)
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    tma0 = box.tma_sweeps()
    e0.record(stream)
    box.run(args.steps, args.cfl)
    e1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    secs = e0.elapsed_time(e1) / 1e3
    tma_per_step = (box.tma_sweeps() - tma0) / args.steps
    box.cfl_dt(args.cfl)               # state still valid after the timed run
    # per-launch figures from a second, traced pass of the same steps from
    # the same state (CUDA events around every launch; the timed pass above
    # has none)
    box.set_state(start)
    del start
    box.profile(args.steps * launches_per_step + 16)
    box.run(args.steps, args.cfl)
    prof = box.profile_read()
    box.profile(0)
    box.cfl_dt(args.cfl)
    secs = max_over_ranks([secs], world)[0]
    value = whole_job_rate(N * args.steps, world, secs)

    # per-kernel roofline of the dominant kernel family
    fam = {"fluid": [prof[k] for k in ("fluid_x", "fluid_y", "fluid_z")],
           "mag": [prof[k] for k in ("mag_x", "mag_y", "mag_z")]}
    tot = {f: sum(ms for _, ms in v) for f, v in fam.items()}
    dom = max(tot, key=tot.get)
    cnt = sum(c for c, _ in fam[dom])
    avg_s = tot[dom] / cnt / 1e3
    achieved = ALGO_BYTES[dom] * N / avg_s / 1e9
    peak, peak_kind = peaks()
    traffic = measured_traffic(dom, n)
    fam_bytes = {"fluid": ALGO_BYTES["fluid"], "mag": ALGO_BYTES["mag"], "transpose": TRANSPOSE_BYTES}
    per_kernel = {k: {"launches": c, "avg_ms": (ms / c if c else None),
                      "GB/s": ((fam_bytes[k.split("_")[0]] * N / (ms / c / 1e3) / 1e9)
                               if c and k != "control" else None)}
                  for k, (c, ms) in prof.items()}
    launches = sum(c for c, _ in prof.values())

    # FP64 diagnostics (compensated sums, max |div b|, min p) of the state:
    # one pass reading the 8 fields (the high faces of a cell are its
    # neighbours' low faces: cache hits), per-launch device time
    diag = None
    if args.diag_reps > 0:
        box.diagnostics()
        box.profile(args.diag_reps + 4)
        for _ in range(args.diag_reps):
            box.diagnostics()
        dc, dms = box.profile_read()["control"]
        box.profile(0)
        d_ms = dms / dc
        d_gbs = DIAG_BYTES * N / (d_ms / 1e3) / 1e9
        diag = {"ms": d_ms, "calls": dc, "algorithmic_bytes_per_cell": DIAG_BYTES, "GB/s": d_gbs,
                "frac": d_gbs / peak, "bound": "hbm"}

    # end-to-end through the C ABI with host buffers: every step copies its
    # input state in from pinned host memory and its result out to pinned
    # host memory.  `value`: the pipelined host API (mhd_submit/mhd_drain:
    # step k overlaps the input copy of k+1 and the output copy of k-1);
    # `sync`: set_state / run / get_state one after the other.
    e2e = None
    if args.e2e_steps > 0:
        out_host = torch.empty_like(host).pin_memory()
        box.submit(host, out_host, 1, args.cfl)   # warm-up (allocates the staging copies)
        box.drain()
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        w0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            box.submit(host, out_host, 1, args.cfl)
        box.drain()
        torch.cuda.synchronize()
        es = time.perf_counter() - w0
        box.set_state(host)
        box.run(1, args.cfl)
        box.get_state(out_host)
        torch.cuda.synchronize()
        w1 = time.perf_counter()
        for _ in range(args.e2e_steps):
            box.set_state(host)          # H2D of the 8 fields
            box.run(1, args.cfl)         # CFL + 12 sweeps
            box.get_state(out_host)      # D2H of the 8 fields (synchronises)
        torch.cuda.synchronize()
        ss = time.perf_counter() - w1
        link = host_link_rate(host, out_host)
        es, ss = max_over_ranks([es, ss], world)
        e2e = {"value": whole_job_rate(N * args.e2e_steps, world, es), "unit": UNIT,
               "h2d_bytes_per_step": 8 * 4 * N, "d2h_bytes_per_step": 8 * 4 * N,
               "ms_per_step": 1e3 * es / args.e2e_steps,
               "api": "mhd_submit x steps + mhd_drain (pinned host in/out, wall clock)",
               "sync": {"value": whole_job_rate(N * args.e2e_steps, world, ss),
                        "ms_per_step": 1e3 * ss / args.e2e_steps,
                        "api": "mhd_set_state + mhd_run(1) + mhd_get_state per step"}}
        # the host link bounds the pipelined API: 32 bytes per cell each way
        bound = world * link * 1e9 / 32.0
        e2e["link_bound"] = {"gbs_each_way": link, "value": bound, "unit": UNIT,
                             "frac": e2e["value"] / bound,
                             "how": "the same 8 fields copied host->device and "
                                    "device->host at once on two streams (best of 2)"}

    ens_out = None
    if args.ensemble_steps > 0:
        box.close()
        torch.cuda.empty_cache()
        ens_out = ensemble_leg(args, world)

    learned_out = None
    if args.learned_reps > 0:
        learned_out = learned_leg(args)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(args.cpu_sample, args.seed, args.cfl)

    # the same kernel against the instruction issue rate: warp instructions
    # per cell (ncu, committed capture) x cells / launch time, against one
    # warp instruction per cycle on each of the 4 schedulers of every SM at
    # the median SM clock sampled during the timed region
    issue = None
    ipc = measured_issue(dom)
    if ipc:
        mhz = (clk or {}).get("sm_mhz") or (clk or {}).get("sm_max_mhz")
        if mhz:
            sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
            ach = ipc * N / avg_s
            pk = sms * 4 * mhz * 1e6
            issue = {"unit": "warp instructions/s", "achieved": ach, "peak": pk, "frac": ach / pk,
                     "warp_instructions_per_cell": ipc,
                     "peak_basis": f"{sms} SMs x 4 schedulers x 1 warp instruction/cycle x {mhz:.0f} MHz"}

    if rank == 0:
        out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps,
               "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
               "data": "synthetic",
               "config": {"workload": f"decaying MHD turbulence {n}^3, "
                                      f"{'periodic' if not bcs else 'non-periodic ' + ','.join(sorted(bcs))}",
                          "n": n, "seed": args.seed, "cfl": args.cfl,
                          "step": "CFL + 6 fluid + 6 magnetic sweeps (x,y,z then z,y,x)",
                          "scheme": {"limiter": args.limiter, "freezing": args.freezing},
                          "xpath": args.xpath or "auto",
                          "fusion": bool(args.fusion),
                          "tma_staged_sweeps_per_step": tma_per_step,
                          **({"boundaries": bcs, "interior_cells": int(np.prod([n - 8 if a in bcs else n for a in "xyz"]))}
                             if bcs else {}),
                          **({"mach": args.mach, "beta": args.beta} if (args.mach, args.beta) != (1.0, 1.0) else {}),
                          "segments": args.seg or "auto",
                          "l2": f"state {32 * N / 1e9:.1f} GB per copy > L2 (no flush needed)",
                          "parallelism": f"replicas x{world}"},
               "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                            "frac": achieved / peak, "traffic": traffic, "kernel": f"{dom} sweep",
                            "algorithmic_bytes_per_cell": ALGO_BYTES[dom],
                            "peak_kind": peak_kind, "issue": issue},
               "step_roofline": {"model_bytes_per_cell": STEP_BYTES,
                                 "achieved_GBps": STEP_BYTES * N * args.steps / secs / 1e9,
                                 "frac": STEP_BYTES * N * args.steps / secs / 1e9 / peak},
               "per_kernel": per_kernel,
               "gpu_launches": launches,
               "precision": precision_record(),
               "clocks": clk,
               "e2e": e2e,
               "diagnostics": diag,
               "cpu_baseline": cpu,
               "ensemble": ens_out,
               "learned_correction": learned_out}
        print(json.dumps(out), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    box.close()
    return 0


def run_fp64(args, rank, world, local):
    """The FP64 path (an ablation of the paper's FP32 computation): the same
    workload and step, every operation in IEEE double; the timestep through
    the host (one synchronisation per step).  CUDA events around the steps."""
    import torch

    from paper_1004_1680_gb300 import initial_conditions as ic
    from paper_1004_1680_gb300 import mhd
    torch.cuda.set_device(local)
    n = args.size
    st = ic.turbulence((n, n, n), seed=args.seed, mach=args.mach, beta=args.beta, device="cuda",
                       dtype=torch.float64)
    box = mhd.Box64(n, n, n)
    box.set_state(st)
    del st
    torch.cuda.empty_cache()
    box.run(args.warmup, args.cfl)
    stream = torch.cuda.current_stream()
    clocks = ClockSampler(None)
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    box.run(args.steps, args.cfl)
    e1.record(stream)
    torch.cuda.synchronize()
    secs = e0.elapsed_time(e1) / 1e3
    clk = clocks.stop()
    if rank == 0:
        out = {"metric": METRIC, "value": n ** 3 * args.steps / secs, "unit": UNIT, "n_gpus": 1,
               "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps,
               "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
               "data": "synthetic",
               "config": {"workload": f"decaying MHD turbulence {n}^3, periodic, FP64 path", "n": n,
                          "seed": args.seed, "cfl": args.cfl},
               "clocks": clk, "e2e": None}
        print(json.dumps(out), flush=True)
    box.close()
    return 0


def run_shard(args, rank, world, local):
    """One periodic box of --size^3 cells cut into z-slabs, one per rank (GPU):
    every step exchanges 16 halo planes of the 8 fields with both z
    neighbours (NCCL), agrees on the CFL timestep (allreduce min) and runs
    the library's step on the slab box.  Whole-box cell-updates/s over the
    slowest rank's time."""
    import torch

    from paper_1004_1680_gb300 import initial_conditions as ic
    from paper_1004_1680_gb300 import slab
    torch.cuda.set_device(local)
    if world > 1:
        torch.distributed.init_process_group("nccl")
    n = args.size
    L = slab.SlabLayout((n, n, n), world, rank)
    st = ic.turbulence((n, n, n), seed=args.seed, mach=args.mach, beta=args.beta, device="cuda",
                       dtype=torch.float32)
    box = slab.make_box(L)
    box.set_state(L.cut(st))
    del st
    torch.cuda.empty_cache()
    ex = slab.SlabExchange(L)
    get = box.get_planes
    put = box.set_planes

    def step():
        ex.exchange(get, put)
        box.step(ex.agree_dt(box.cfl_dt(args.cfl), device="cuda"))
    for _ in range(args.warmup):
        step()
    clocks = ClockSampler(None)
    clocks.start()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    torch.cuda.synchronize()
    secs = time.perf_counter() - t0
    clk = clocks.stop()
    secs = max_over_ranks([secs], world)[0]
    if rank == 0:
        out = {"metric": METRIC, "value": n ** 3 * args.steps / secs, "unit": UNIT, "n_gpus": world,
               "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps,
               "higher_is_better": True, "scaling": "strong", "vs_baseline": None, "dtype": "f32",
               "data": "synthetic",
               "config": {"workload": f"decaying MHD turbulence {n}^3, periodic, one box in z-slabs",
                          "n": n, "seed": args.seed, "cfl": args.cfl,
                          "slab": {"own_planes": L.own, "halo_planes": L.halo, "local_dims": L.local_dims},
                          "parallelism": f"z-slabs x{world}",
                          "timing": "wall clock around the steps (host-driven exchange), max over ranks"},
               "clocks": clk, "e2e": None}
        print(json.dumps(out), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    box.close()
    return 0


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.shard:
        return run_shard(args, rank, world, local)
    if args.fp64:
        return run_fp64(args, rank, world, local)
    return run_ours(args, rank, world, local)


if __name__ == "__main__":
    sys.exit(main())
