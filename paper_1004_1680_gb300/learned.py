"""Learned coarse-grid correction (an extension; not in the paper).

A 4-layer 3x3x3 periodic CNN (8 -> 32 -> 32 -> 32 -> 8 channels, ReLU between
layers, BF16 operands with FP32 accumulation on the tcgen05 tensor cores,
FP32 master weights) maps a coarse state to a correction that is applied
after each coarse step:
  * channels 0-4 give the corrections of rho, m, e, with their box means
    removed (mass, momentum and energy stay conserved);
  * channels 5-7 give an edge vector potential whose discrete curl is the
    face-field correction (div b stays zero);
  * mhd_correct clips the correction so that rho and the thermal energy stay
    positive.
Training pairs come from the solver itself: input R(U_f(t)) (a 256^3 state
restricted to 64^3), target R(U_f(t + dt)) - C(R(U_f(t))) where C is one
coarse step of length dt and the fine run advances by the same dt.  With
rollout > 1 a pair's input may also be a coarse state that has run freely
for a few steps from R(U_f) (target: R(U_f) at the end of the next step
minus that step's result), so that the network also sees the drift that a
coarse run accumulates.  The scale of the applied correction is chosen on
validation seeds (choose_alpha), never on the seeds the comparison uses.

Every arithmetic step runs in the CUDA library (convolutions, projection,
loss, Adam, restriction, solver); this module sequences the calls.
"""
from __future__ import annotations

import math
import time
from dataclasses import dataclass, field

import numpy as np
import torch

from . import initial_conditions as ic
from . import mhd

LAYERS = [(8, 32), (32, 32), (32, 32), (32, 8)]


class CorrectionNet:
    def __init__(self, seed: int = 0, device="cuda", out_scale: float = 0.1):
        g = torch.Generator().manual_seed(seed)
        self.W, self.b = [], []
        for li, (ci, co) in enumerate(LAYERS):
            std = math.sqrt(2.0 / (ci * 27))
            if li == len(LAYERS) - 1:
                std *= out_scale           # start close to "no correction"
            self.W.append((torch.randn(co, ci, 3, 3, 3, generator=g) * std).to(device))
            self.b.append(torch.zeros(co, device=device))
        self.params = self.W + self.b
        self.m = [torch.zeros_like(p) for p in self.params]
        self.v = [torch.zeros_like(p) for p in self.params]
        self.step_count = 0
        self.repack()

    def repack(self):
        self.img = [mhd.conv_pack(w) for w in self.W]
        self.imgT = [mhd.conv_pack(w, transpose=True) for w in self.W]

    def forward(self, x: torch.Tensor, n):
        """x: (cells, 8) BF16 -> y (cells, 8) FP32 and the activations."""
        acts = [x]
        h = x
        for li, (ci, co) in enumerate(LAYERS):
            last = li == len(LAYERS) - 1
            hb, hf = mhd.conv3d(h, self.img[li], n, ci, co, bias=self.b[li], relu=not last,
                                out_bf16=not last, out_f32=last)
            h = hf if last else hb
            if not last:
                acts.append(h)
        return h, acts

    def backward(self, gy: torch.Tensor, acts, n):
        """gy: (cells, 8) BF16 gradient of the loss w.r.t. y; fills self.grads."""
        self.grads = [torch.zeros_like(p) for p in self.params]
        g = gy
        L = len(LAYERS)
        for li in range(L - 1, -1, -1):
            ci, co = LAYERS[li]
            mhd.conv3d_wgrad(acts[li], g, n, ci, co, self.grads[li].view(-1), self.grads[L + li])
            if li > 0:
                g, _ = mhd.conv3d(g, self.imgT[li], n, co, ci, flip=True, mask=acts[li])

    def adam(self, lr: float):
        self.step_count += 1
        for p, gr, m, v in zip(self.params, self.grads, self.m, self.v):
            mhd.adam(p.view(-1), gr.view(-1), m.view(-1), v.view(-1), lr, self.step_count)
        self.repack()

    def state_dict(self):
        return {"W": [w.cpu() for w in self.W], "b": [b.cpu() for b in self.b]}


@dataclass
class Norm:
    """Per-field input normalisation and output scales."""
    mu: list
    inv_sigma: list
    out_scale: list            # 5 cell scales + the edge-potential scale
    loss_weight: list = field(default_factory=list)


class Corrector:
    """Network + normalisation: correction of a coarse state."""

    def __init__(self, net: CorrectionNet, norm: Norm, n, alpha: float = 1.0):
        """alpha scales the applied correction (the projection is linear, so
        it scales the output scales)."""
        self.net, self.norm, self.n = net, norm, n
        self.out_scale = [alpha * x for x in norm.out_scale]
        cells = n[0] * n[1] * n[2]
        dev = net.W[0].device
        self.x = torch.empty((cells, 8), dtype=torch.bfloat16, device=dev)
        self.d = torch.empty((8, n[2], n[1], n[0]), dtype=torch.float32, device=dev)
        self.sums = torch.empty(5, dtype=torch.float64, device=dev)
        self.scratch = torch.empty(cells, dtype=torch.float32, device=dev)

    def predict(self, state: torch.Tensor) -> torch.Tensor:
        """Correction for the coarse step that starts from `state` (the
        network input is the state before the step, as in the training pairs)."""
        mhd.cnn_normalize(state, self.norm.mu, self.norm.inv_sigma, out=self.x)
        y, _ = self.net.forward(self.x, self.n)
        return mhd.cnn_project(y, self.n, self.out_scale, out=self.d, sums=self.sums)

    def apply(self, stepped: torch.Tensor, d: torch.Tensor, nclip=None):
        """Add a predicted correction to the state after the coarse step."""
        mhd.correct(stepped, d, scratch=self.scratch, nclip=nclip)


# --------------------------------------------------------------------------
# training data from the solver

def fine_substeps(fine: mhd.Box, dt: float, cfl: float) -> int:
    return max(1, int(math.ceil(dt / fine.cfl_dt(cfl) - 1e-9)))


def advance_fine(fine: mhd.Box, dt: float, cfl: float):
    k = fine_substeps(fine, dt, cfl)
    for _ in range(k):
        fine.step(dt / k)


def generate_pairs(seeds, steps_per_seed: int = 1, nf: int = 256, r: int = 4, cfl: float = 0.7,
                   p_floor: float = 1e-3, mach: float = 1.0, beta: float = 1.0, t_max: int = 0,
                   rollout: int = 1, rng_seed: int = 12345, kmin: float = 2.0, kmax: float = 8.0, log=None):
    """Pairs (coarse input, target residual) from a fine run of each seed.

    A seed's fine run gives `steps_per_seed` segments, at coarse step counts
    k drawn without repetition from [0, t_max) and sorted (t_max = 0: the
    first steps_per_seed steps, k = 0, 1, ...); between them the fine run
    takes r of its own CFL steps per coarse step (its cells are r times
    smaller, so a coarse CFL step spans about r fine ones).  A segment
    restricts the fine state to the coarse grid and lets the coarse box run
    `rollout` steps freely next to the fine run; step j of the segment gives
    the pair (coarse state before the step, R(fine after the step) - coarse
    state after the step).  Returns two tensors (P, 8, nc, nc, nc) on the
    GPU."""
    nc = nf // r
    fine = mhd.Box(nf, nf, nf)
    coarse = mhd.Box(nc, nc, nc)
    fine.set_pressure_floor(p_floor)
    coarse.set_pressure_floor(p_floor)
    rng = np.random.default_rng(rng_seed)
    ins, tgts = [], []
    skipped = []
    t0 = time.perf_counter()
    for si, seed in enumerate(seeds):
        st = ic.turbulence((nf, nf, nf), seed=seed, mach=mach, beta=beta, device="cuda", dtype=torch.float32,
                           kmin=kmin, kmax=kmax)
        fine.set_state(st)
        del st
        if t_max > 0:
            ks = np.sort(rng.choice(t_max, size=steps_per_seed, replace=False))
        else:
            ks = np.arange(steps_per_seed)
        k = 0
        seed_ins, seed_tgts = [], []
        try:
            for kt in ks:
                if kt > k:           # r fine CFL steps per coarse step (h is r times smaller)
                    fine.run(int(r * (kt - k)), cfl)
                    k = int(kt)
                fine.cfl_dt(cfl)     # raises if the fine run left the valid states
                coarse.set_state(mhd.restrict(fine.get_state(), r))
                for _ in range(rollout):
                    uc0 = coarse.get_state()
                    dt = coarse.cfl_dt(cfl)
                    coarse.step(dt)
                    uc1 = coarse.get_state()
                    advance_fine(fine, dt, cfl)
                    seed_ins.append(uc0)
                    seed_tgts.append(mhd.restrict(fine.get_state(), r) - uc1)
                    coarse.cfl_dt(cfl)
                k += rollout
        except mhd.MHDError as e:  # an invalid state (p <= 0 or NaN): the seed gives no pairs
            skipped.append(seed)
            if log:
                log(f"seed {seed} skipped: {e}")
            continue
        ins += seed_ins
        tgts += seed_tgts
        if log and (si + 1) % 50 == 0:
            log(f"pairs: {si + 1} seeds, {len(ins)} pairs, {time.perf_counter() - t0:.0f} s")
    fine.close()
    coarse.close()
    generate_pairs.skipped = skipped
    return torch.stack(ins), torch.stack(tgts)


def make_norm(inputs: torch.Tensor, targets: torch.Tensor, nc: int) -> Norm:
    mu = inputs.mean(dim=(0, 2, 3, 4)).tolist()
    sig = inputs.std(dim=(0, 2, 3, 4)).clamp_min(1e-6).tolist()
    ts = targets.std(dim=(0, 2, 3, 4)).clamp_min(1e-12).tolist()
    # edge potential scale: its curl (differences over h = 1/nc) matches the
    # face-field residual scale
    sA = float(np.mean(ts[5:8])) / nc
    out_scale = ts[:5] + [sA]
    weight = [1.0 / (8.0 * t * t * inputs[0, 0].numel()) for t in ts]
    return Norm(mu=mu, inv_sigma=[1.0 / s for s in sig], out_scale=out_scale, loss_weight=weight)


def train(inputs, targets, norm: Norm, epochs: int, lr: float = 1e-3, seed: int = 0, log=None):
    nc = inputs.shape[-1]
    n = (nc, nc, nc)
    net = CorrectionNet(seed=seed)
    corr = Corrector(net, norm, n)
    g = torch.empty_like(corr.d)
    loss = torch.empty(1, dtype=torch.float64, device="cuda")
    gy = torch.empty((nc ** 3, 8), dtype=torch.bfloat16, device="cuda")
    sums = torch.empty(5, dtype=torch.float64, device="cuda")
    P = inputs.shape[0]
    rng = np.random.default_rng(seed)
    history = []
    t0 = time.perf_counter()
    for ep in range(epochs):
        lr_ep = lr * (0.05 + 0.95 * 0.5 * (1.0 + math.cos(math.pi * ep / max(1, epochs))))   # cosine decay
        order = rng.permutation(P)
        tot = 0.0
        for i in order:
            mhd.cnn_normalize(inputs[i], norm.mu, norm.inv_sigma, out=corr.x)
            y, acts = net.forward(corr.x, n)
            d = mhd.cnn_project(y, n, norm.out_scale, out=corr.d, sums=corr.sums)
            mhd.cnn_loss(d, targets[i], norm.loss_weight, g=g, loss=loss)
            mhd.cnn_project_backward(g, norm.out_scale, out=gy, sums=sums)
            net.backward(gy, acts, n)
            net.adam(lr_ep)
            tot += float(loss.item()) if (i == order[-1]) else 0.0
        # epoch loss on a fixed subset (no update)
        ev = 0.0
        sub = range(0, P, max(1, P // 32))
        for i in sub:
            d = corr.predict(inputs[i])
            ev += float(mhd.cnn_loss(d, targets[i], norm.loss_weight, loss=loss).item())
        history.append(ev / len(sub))
        if log:
            log(f"epoch {ep}: loss {history[-1]:.4f} ({time.perf_counter() - t0:.1f} s)")
    return net, history


# --------------------------------------------------------------------------
# evaluation: learned 64^3 vs plain 64^3 / 128^3 against the restricted 256^3

def nrmse(run: torch.Tensor, ref: torch.Tensor) -> np.ndarray:
    d = (run - ref).double()
    rms = torch.sqrt((d ** 2).mean(dim=(1, 2, 3)))
    sd = ref.double().std(dim=(1, 2, 3)).clamp_min(1e-30)
    return (rms / sd).cpu().numpy()


def evaluate(corrector, seed: int, nsteps: int = 200, every: int = 20, nf: int = 256,
             cfl: float = 0.7, p_floor: float = 1e-3, mach: float = 1.0, beta: float = 1.0, nc: int = 64,
             kmin: float = 2.0, kmax: float = 8.0):
    """Errors of learned nc^3, plain nc^3 and plain (2 nc)^3 runs against the
    fine nf^3 run restricted to nc^3 at the same times (all runs follow the
    plain nc^3 run's CFL dt), and GPU times.  (The result keys keep the
    names of the 256^3 -> 64^3 workload: learned64, plain64, plain128.)
    `corrector` is a Corrector, None (no correction), or a list of
    Correctors: then every one of them runs its own learned coarse box next
    to the same reference, under the keys learned64/<i>."""
    st = ic.turbulence((nf, nf, nf), seed=seed, mach=mach, beta=beta, device="cuda", dtype=torch.float32,
                       kmin=kmin, kmax=kmax)
    correctors = corrector if isinstance(corrector, (list, tuple)) else [corrector]
    lkeys = ["learned64"] if not isinstance(corrector, (list, tuple)) else \
        [f"learned64/{i}" for i in range(len(correctors))]
    boxes = {"ref": mhd.Box(nf, nf, nf), "plain64": mhd.Box(nc, nc, nc), "plain128": mhd.Box(2 * nc, 2 * nc, 2 * nc)}
    for k in lkeys:
        boxes[k] = mhd.Box(nc, nc, nc)
    for b in boxes.values():
        b.set_pressure_floor(p_floor)
    boxes["ref"].set_state(st)
    boxes["plain64"].set_state(mhd.restrict(st, nf // nc))
    for k in lkeys:
        boxes[k].set_state(mhd.restrict(st, nf // nc))
    boxes["plain128"].set_state(mhd.restrict(st, nf // (2 * nc)))
    del st
    ev = {k: (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for k in boxes}
    gpu_ms = {k: 0.0 for k in boxes}
    errs = {k: [] for k in ["plain64", "plain128"] + lkeys}
    lstate = boxes[lkeys[0]].get_state()
    nclip = torch.zeros(1, dtype=torch.int32, device="cuda")
    cmap = dict(zip(lkeys, correctors))
    for s in range(1, nsteps + 1):
        dt = boxes["plain64"].cfl_dt(cfl)
        for k, b in boxes.items():
            ev[k][0].record()
            if k == "ref":
                advance_fine(b, dt, cfl)
            elif k == "plain128":
                kk = max(2, fine_substeps(b, dt, cfl))
                for _ in range(kk):
                    b.step(dt / kk)
            elif k in cmap:
                c = cmap[k]
                if c is not None:
                    b.get_state(out=lstate)
                    d = c.predict(lstate)
                b.step(dt)
                if c is not None:
                    b.get_state(out=lstate)
                    c.apply(lstate, d, nclip=nclip)
                    b.set_state(lstate)   # (its own time and CFL rate are not used)
            else:
                b.step(dt)
            ev[k][1].record()
            torch.cuda.synchronize()
            gpu_ms[k] += ev[k][0].elapsed_time(ev[k][1])
        if s % every == 0:
            ref = mhd.restrict(boxes["ref"].get_state(), nf // nc)
            errs["plain64"].append(nrmse(boxes["plain64"].get_state(), ref))
            for k in lkeys:
                errs[k].append(nrmse(boxes[k].get_state(), ref))
            errs["plain128"].append(nrmse(mhd.restrict(boxes["plain128"].get_state(), 2), ref))
    t = boxes["plain64"].time()
    for b in boxes.values():
        b.close()
    return {k: np.array(v) for k, v in errs.items()}, gpu_ms, t, int(nclip.item())


def evaluate_safe(corrector, seed: int, log=None, **kw):
    """evaluate(), or None if one of the runs leaves the valid states (the
    seed is then left out and counted)."""
    try:
        return evaluate(corrector, seed, **kw)
    except mhd.MHDError as e:
        if log:
            log(f"seed {seed} left out: {e}")
        return None


def choose_alpha(net: CorrectionNet, norm: Norm, seeds, alphas=(0.0, 0.25, 0.5, 0.75, 1.0), nsteps: int = 200,
                 nf: int = 256, nc: int = 64, every: int = 20, log=None, **kw):
    """The scale of the applied correction with the lowest mean error on
    validation seeds (alpha 0 is the plain coarse run): every alpha runs
    next to the same reference runs.  Returns (best alpha, {alpha: mean
    NRMSE})."""
    cs = [Corrector(net, norm, (nc, nc, nc), alpha=a) for a in alphas]
    tot = np.zeros(len(alphas))
    used = 0
    for seed in seeds:
        r = evaluate_safe(cs, seed, log=log, nsteps=nsteps, nf=nf, nc=nc, every=min(every, nsteps), **kw)
        if r is None:
            continue
        errs = r[0]
        used += 1
        for i in range(len(alphas)):
            tot[i] += errs[f"learned64/{i}"].mean()
        if log:
            log(f"validation seed {seed}: " + " ".join(f"{a}:{errs[f'learned64/{i}'].mean():.4f}"
                                                      for i, a in enumerate(alphas)))
    means = {a: float(t / max(used, 1)) for a, t in zip(alphas, tot)}
    return min(means, key=means.get), means
