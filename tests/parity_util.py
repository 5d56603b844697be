"""Shared helpers of the GPU-vs-oracle parity tests."""
import math

import numpy as np
import torch

import oracle

G = 5.0 / 3.0


def field_scales(s0: np.ndarray, gamma: float = G) -> np.ndarray:
    """Per-field error scales S_f (normalisation of the max relative error):
    S_rho = mean rho, S_m = mean rho * rms fast speed, S_e = mean e,
    S_b = rms |b|.  A perturbation far below the background (a 1e-6 wave on
    O(1) fields) is thus measured against the background, not against
    itself, since FP32 cannot resolve it better than its own rounding."""
    rho = s0[0]
    p = oracle.pressure(s0, gamma)
    b2 = sum((0.5 * (s0[5 + d] + np.roll(s0[5 + d], -1, axis=2 - d))) ** 2 for d in range(3))
    cref = math.sqrt(float(np.mean((gamma * np.maximum(p, 0) + b2) / rho)))
    rbar = float(np.mean(rho))
    brms = math.sqrt(float(np.mean(s0[5] ** 2 + s0[6] ** 2 + s0[7] ** 2)))
    return np.array([rbar, rbar * cref, rbar * cref, rbar * cref, float(np.mean(s0[4])),
                     brms, brms, brms])


def rel_err(gpu: np.ndarray, orc: np.ndarray, S: np.ndarray) -> np.ndarray:
    """err_f = max |gpu - oracle| / max(max |oracle_f|, S_f), per field (an
    identically zero field, e.g. b in a hydrodynamic tube, is compared
    absolutely)."""
    out = np.zeros(8)
    for q in range(8):
        den = max(float(np.max(np.abs(orc[q]))), float(S[q])) or 1.0
        out[q] = float(np.max(np.abs(gpu[q].astype(np.float64) - orc[q]))) / den
    return out


def l1_rel(gpu: np.ndarray, orc: np.ndarray, S: np.ndarray) -> np.ndarray:
    """Mean absolute difference over the scale, per field."""
    out = np.zeros(8)
    for q in range(8):
        den = max(float(np.mean(np.abs(orc[q]))), float(S[q])) or 1.0
        out[q] = float(np.mean(np.abs(gpu[q].astype(np.float64) - orc[q]))) / den
    return out


def to_gpu(state64: torch.Tensor) -> torch.Tensor:
    return state64.to(torch.float32).contiguous().cuda()


def from_gpu(t: torch.Tensor) -> np.ndarray:
    return t.detach().cpu().numpy().astype(np.float64)


def sub_block(s: np.ndarray, lo, size):
    """Periodic sub-block of a state: cells lo[d] .. lo[d]+size[d]-1 (wrapped)."""
    idx = [np.arange(lo[d], lo[d] + size[d]) % s.shape[3 - d] for d in range(3)]
    return np.ascontiguousarray(s[:, idx[2]][:, :, idx[1]][:, :, :, idx[0]])
