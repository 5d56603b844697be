"""Seeded synthetic initial states for the MHD grid update.

This module builds inputs only: it holds none of the update's arithmetic.  It
serves both the CUDA path and the FP64 oracle, so that the two are compared on
identical states.

Conventions (shared with the library):
  * the domain is the periodic unit cube, n = (nx, ny, nz), h_d = 1/n_d;
  * a state is float64 (or float32) of shape (8, nz, ny, nx) holding
    rho, m_x, m_y, m_z, e, b_x, b_y, b_z, x fastest;
  * b_d[k, j, i] is the mean normal field over the low face of cell (i, j, k)
    along d;
  * b is in units where 4*pi is absorbed (Section II.A), so
    e = p/(gamma-1) + rho v^2/2 + |b_c|^2/2, with b_c the mean of a cell's two
    faces.

Every field is set from band-limited Fourier modes evaluated as exact cell,
face or edge averages, and the magnetic field is the discrete curl of an edge
vector potential, so div b is zero up to rounding by construction.
"""
from __future__ import annotations

import math
from typing import Sequence

import numpy as np
import torch

GAMMA = 5.0 / 3.0


# --------------------------------------------------------------------------
# band-limited evaluation

def eval_modes(K: np.ndarray, C: np.ndarray, n: Sequence[int], offset=(0.5, 0.5, 0.5),
               average=(True, True, True), device="cpu", out_dtype=torch.float64,
               slab: int = 64) -> torch.Tensor:
    """Re sum_m C_m exp(2 pi i K_m . x) on an nx*ny*nz grid.

    K: (M, 3) integer wave vectors (x, y, z); C: (M,) complex coefficients.
    offset[a]: sample position in cell units along axis a (0.5 = cell centre,
    0 = low face).  average[a]: if true, the value is the exact mean over the
    cell width along a (a factor sinc(pi k_a / n_a) per mode) instead of a
    point value.  Returns a tensor of shape (nz, ny, nx).
    """
    K = np.asarray(K, dtype=np.int64).reshape(-1, 3)
    C = np.asarray(C, dtype=np.complex128).reshape(-1)
    nx, ny, nz = (int(v) for v in n)
    kmax = int(np.max(np.abs(K))) if K.size else 0
    w = 2 * kmax + 1
    cube = np.zeros((w, w, w), dtype=np.complex128)            # [kz, ky, kx]
    np.add.at(cube, (K[:, 2] + kmax, K[:, 1] + kmax, K[:, 0] + kmax), C)

    def basis(na, off, avg):
        k = np.arange(-kmax, kmax + 1)
        x = (np.arange(na) + off) / na
        E = np.exp(2j * np.pi * np.outer(x, k))                  # (na, w)
        if avg:
            E = E * np.sinc(k / na)[None, :]                     # np.sinc(t)=sin(pi t)/(pi t)
        return torch.from_numpy(E).to(device)

    Ex = basis(nx, offset[0], average[0])
    Ey = basis(ny, offset[1], average[1])
    Ez = basis(nz, offset[2], average[2])
    cub = torch.from_numpy(cube).to(device)
    G = torch.einsum("zyk,ik->zyi", cub, Ex)                    # (w, w, nx)
    H = torch.einsum("zyi,jy->zji", G, Ey).reshape(w, ny * nx)  # (w, ny*nx)
    out = torch.empty((nz, ny, nx), dtype=out_dtype, device=device)
    for k0 in range(0, nz, slab):
        k1 = min(nz, k0 + slab)
        out[k0:k1] = (Ez[k0:k1] @ H).real.reshape(k1 - k0, ny, nx).to(out_dtype)
    return out


def curl_edges(Ax: torch.Tensor, Ay: torch.Tensor, Az: torch.Tensor, n: Sequence[int]):
    """Face field b = discrete curl of an edge vector potential.

    A_x[k, j, i] is the mean of A_x along the x-edge at (x_i, y_{j-1/2}, z_{k-1/2}),
    A_y at (x_{i-1/2}, y_j, z_{k-1/2}), A_z at (x_{i-1/2}, y_{j-1/2}, z_k).
    By Stokes' theorem each face value is the circulation around the face
    divided by its area, so the discrete divergence of b vanishes identically.
    """
    nx, ny, nz = n

    def up(a, axis):  # value at index + 1 along a numpy axis (periodic)
        return torch.roll(a, shifts=-1, dims=axis)

    bx = (up(Az, 1) - Az) * ny - (up(Ay, 0) - Ay) * nz
    by = (up(Ax, 0) - Ax) * nz - (up(Az, 2) - Az) * nx
    bz = (up(Ay, 2) - Ay) * nx - (up(Ax, 1) - Ax) * ny
    return bx, by, bz


def cell_centred(b: torch.Tensor, d: int) -> torch.Tensor:
    """Mean of the low and high face of each cell along axis d."""
    return 0.5 * (b + torch.roll(b, shifts=-1, dims=2 - d))


def assemble(rho, v, p, b, gamma=GAMMA, dtype=torch.float64) -> torch.Tensor:
    """Conserved state from primitives: m = rho v, e = p/(gamma-1) + m.v/2 + |b_c|^2/2."""
    rho = torch.as_tensor(rho, dtype=torch.float64)
    shape = rho.shape
    dev = rho.device
    out = torch.empty((8,) + tuple(shape), dtype=torch.float64, device=dev)
    out[0] = rho
    for a in range(3):
        out[1 + a] = rho * torch.as_tensor(v[a], dtype=torch.float64, device=dev)
    bb = [torch.as_tensor(b[a], dtype=torch.float64, device=dev).expand(shape) for a in range(3)]
    b2 = sum(cell_centred(bb[a], a) ** 2 for a in range(3))
    kin = 0.5 * (out[1] ** 2 + out[2] ** 2 + out[3] ** 2) / rho
    out[4] = torch.as_tensor(p, dtype=torch.float64, device=dev) / (gamma - 1.0) + kin + 0.5 * b2
    for a in range(3):
        out[5 + a] = bb[a]
    return out.to(dtype)


def _full(n, value, device="cpu"):
    nx, ny, nz = n
    return torch.full((nz, ny, nx), float(value), dtype=torch.float64, device=device)


# --------------------------------------------------------------------------
# test problems

def uniform(n, rho=1.0, v=(0.0, 0.0, 0.0), p=1.0, b=(0.0, 0.0, 0.0), gamma=GAMMA):
    """Constant state."""
    return assemble(_full(n, rho), [_full(n, x) for x in v], _full(n, p),
                    [_full(n, x) for x in b], gamma)


def _unit(v):
    v = np.asarray(v, dtype=np.float64)
    return v / np.linalg.norm(v)


def _perp(khat):
    """A fixed unit vector perpendicular to khat: the first of (1,-1,0), (0,1,0),
    (0,0,1) with a large enough perpendicular part, made perpendicular."""
    for trial in ([1.0, -1.0, 0.0], [0.0, 1.0, 0.0], [0.0, 0.0, 1.0]):
        t = np.asarray(trial)
        e = t - khat * np.dot(t, khat)
        if np.linalg.norm(e) > 0.5:
            return _unit(e)
    raise ValueError("no perpendicular found")


def plane_wave_potential(n, k_int, w, phase_fn="sin"):
    """Edge-averaged A = w * sin(k.x) / |k| for integer wave vector k_int (k = 2 pi k_int);
    its curl is cos(k.x) (khat x w) exactly on faces."""
    k_int = np.asarray(k_int, dtype=np.int64)
    kabs = 2 * math.pi * float(np.linalg.norm(k_int))
    K = k_int[None, :]
    out = []
    # A_x on x-edges: centre in x, low face in y and z; mean along x only
    offs = [((0.5, 0.0, 0.0), (True, False, False)),
            ((0.0, 0.5, 0.0), (False, True, False)),
            ((0.0, 0.0, 0.5), (False, False, True))]
    for a in range(3):
        coef = -1j * w[a] / kabs          # Re(-i c e^{i t}) = c sin t
        out.append(eval_modes(K, [coef], n, offset=offs[a][0], average=offs[a][1]))
    return out


def _cos_cells(n, k_int, amp):
    """Cell averages of amp * cos(2 pi k_int . x)."""
    return eval_modes(np.asarray(k_int)[None, :], [amp], n)


def alfven_wave(n, k_int=(1, 1, 1), amp=1e-6, rho=1.0, p=0.1, B0=1.0, gamma=GAMMA,
                e_perp=None):
    """Linear Alfven wave travelling along +khat with B0 along khat.

    dv = amp * e_perp * cos(k.x), db = -sqrt(rho) * dv (so the perturbation
    translates along khat at v_A = B0/sqrt(rho)); b is the curl of an edge
    potential.  Returns the state and a dict with the wave's parameters.
    """
    khat = _unit(k_int)
    e = _perp(khat) if e_perp is None else _unit(e_perp)
    dv = _cos_cells(n, k_int, amp)
    v = [dv * e[a] for a in range(3)]
    w = -math.sqrt(rho) * amp * np.cross(e, khat)
    A = plane_wave_potential(n, k_int, w)
    db = curl_edges(*A, n)
    b = [db[a] + B0 * khat[a] for a in range(3)]
    st = assemble(_full(n, rho), v, _full(n, p), b, gamma)
    info = dict(khat=khat, e_perp=e, v_A=B0 / math.sqrt(rho),
                period=1.0 / (float(np.linalg.norm(k_int)) * B0 / math.sqrt(rho)))
    return st, info


def fast_wave(n, k_int=(1, 0, 0), amp=1e-6, rho=1.0, p=0.1, B0=(0.0, 1.0, 0.0),
              gamma=GAMMA, v0=0.0):
    """Linear fast magnetosonic wave along +khat with B0 perpendicular to khat,
    optionally carried by a uniform flow v0 * khat (Galilean boost).

    c_f = sqrt((gamma p + |B0|^2)/rho); drho/rho = amp cos(k.x),
    dv = amp c_f khat cos, dp = gamma p amp cos, db = amp B0 cos; the pattern
    translates at c_f + v0 along khat.
    """
    khat = _unit(k_int)
    B0 = np.asarray(B0, dtype=np.float64)
    if abs(np.dot(B0, khat)) > 1e-12:
        raise ValueError("B0 must be perpendicular to k")
    cf = math.sqrt((gamma * p + float(np.dot(B0, B0))) / rho)
    c = _cos_cells(n, k_int, 1.0)
    r = rho * (1.0 + amp * c)
    v = [(v0 + amp * cf * c) * khat[a] for a in range(3)]
    pp = p * (1.0 + gamma * amp * c)
    w = amp * np.cross(B0, khat)
    A = plane_wave_potential(n, k_int, w)
    db = curl_edges(*A, n)
    b = [db[a] + B0[a] for a in range(3)]
    st = assemble(r, v, pp, b, gamma)
    info = dict(khat=khat, c_f=cf, period=1.0 / (float(np.linalg.norm(k_int)) * (cf + v0)))
    return st, info


def sod(n, axis=0, left=(1.0, 1.0), right=(0.125, 0.1), gamma=GAMMA):
    """B = 0 shock tube along `axis`: (rho, p) = left for x_axis < 0.5, right otherwise.
    On the periodic box a mirrored Riemann problem also sits at x_axis = 0."""
    nx, ny, nz = n
    na = n[axis]
    xc = (torch.arange(na, dtype=torch.float64) + 0.5) / na
    lefty = (xc < 0.5).to(torch.float64)
    shape = [1, 1, 1]
    shape[2 - axis] = na
    lefty = lefty.reshape(shape).expand(nz, ny, nx)
    rho = right[0] + (left[0] - right[0]) * lefty
    p = right[1] + (left[1] - right[1]) * lefty
    zero = _full(n, 0.0)
    return assemble(rho, [zero, zero, zero], p, [zero, zero, zero], gamma)


def orszag_tang(n, gamma=GAMMA):
    """3-D Orszag-Tang-style vortex: rho = 25/(36 pi), p = 5/(12 pi),
    v = (-sin 2pi y, sin 2pi x, 0.1 sin 2pi z),
    b = (-sin 2pi y, sin 4pi x, 0)/sqrt(4 pi) from
    A_z = (cos 4pi x / (4pi) + cos 2pi y / (2pi)) / sqrt(4 pi)."""
    rho = _full(n, 25.0 / (36.0 * math.pi))
    p = _full(n, 5.0 / (12.0 * math.pi))
    # -sin t = Re(i e^{i t}); sin t = Re(-i e^{i t})
    vx = eval_modes([[0, 1, 0]], [1j], n)
    vy = eval_modes([[1, 0, 0]], [-1j], n)
    vz = eval_modes([[0, 0, 1]], [-0.1j], n)
    s = 1.0 / math.sqrt(4.0 * math.pi)
    off_z, avg_z = (0.0, 0.0, 0.5), (False, False, True)
    Az = eval_modes([[2, 0, 0], [0, 1, 0]], [s / (4 * math.pi), s / (2 * math.pi)], n,
                    offset=off_z, average=avg_z)
    zero = _full(n, 0.0)
    b = curl_edges(zero, zero, Az, n)
    return assemble(rho, [vx, vy, vz], p, list(b), gamma)


def _band_modes(rng, kmin=2.0, kmax=8.0):
    r = int(math.floor(kmax))
    g = np.arange(-r, r + 1)
    K = np.stack(np.meshgrid(g, g, g, indexing="ij"), axis=-1).reshape(-1, 3)
    kk = np.linalg.norm(K, axis=1)
    K = K[(kk >= kmin) & (kk <= kmax)]
    return K


def _solenoidal_coeffs(rng, K, slope_amp):
    """Complex Gaussian 3-vectors per mode, projected perpendicular to k,
    scaled by |k|^slope_amp."""
    M = K.shape[0]
    c = rng.standard_normal((M, 3)) + 1j * rng.standard_normal((M, 3))
    kh = K / np.linalg.norm(K, axis=1, keepdims=True)
    c = c - kh * np.sum(c * kh, axis=1, keepdims=True)
    return c * (np.linalg.norm(K, axis=1) ** slope_amp)[:, None]


def turbulence(n, seed=0, mach=1.0, beta=1.0, rho=1.0, p=1.0, gamma=GAMMA,
               device="cpu", dtype=torch.float32, kmin=2.0, kmax=8.0):
    """Decaying-turbulence initial state.

    Shell spectrum E(k) ~ k^-2 for kmin <= |k|/(2 pi) <= kmax (per-mode
    |v_k|^2 ~ k^-4), Gaussian random phases from np.random.default_rng(seed),
    solenoidal v rescaled to rms |v| = mach * sqrt(gamma p / rho); b = curl A
    with A drawn from the same band (|b_k|^2 ~ k^-4 as well), rescaled so that
    beta = 2 p / <|b_c|^2>.  Uniform rho and p.
    """
    rng = np.random.default_rng(seed)
    K = _band_modes(rng, kmin, kmax)
    cv = _solenoidal_coeffs(rng, K, -2.0)
    ca = _solenoidal_coeffs(rng, K, -3.0)
    v = [eval_modes(K, cv[:, a], n, device=device) for a in range(3)]
    vrms = math.sqrt(float(sum((va ** 2).mean() for va in v)))
    sv = mach * math.sqrt(gamma * p / rho) / vrms
    v = [va * sv for va in v]
    offs = [((0.5, 0.0, 0.0), (True, False, False)),
            ((0.0, 0.5, 0.0), (False, True, False)),
            ((0.0, 0.0, 0.5), (False, False, True))]
    A = [eval_modes(K, ca[:, a] / (2 * math.pi), n, offset=offs[a][0], average=offs[a][1],
                    device=device) for a in range(3)]
    b = list(curl_edges(*A, n))
    b2 = float(sum((cell_centred(b[a], a) ** 2).mean() for a in range(3)))
    sb = math.sqrt(2.0 * p / beta / b2)
    b = [ba * sb for ba in b]
    rr = torch.full_like(v[0], rho)
    pp = torch.full_like(v[0], p)
    return assemble(rr, v, pp, b, gamma, dtype=dtype)


def ensemble_specs(nbox=256, seed=2024, sizes=(32, 48, 64, 96)):
    """Per-box (dims, seed, mach, beta) for the uneven-box ensemble: per-axis
    size uniform in `sizes`, box b seeded 1000+b, Mach ~ U[0.5, 2],
    beta log-uniform in [0.3, 3]."""
    rng = np.random.default_rng(seed)
    dims = rng.choice(np.asarray(sizes), size=(nbox, 3))
    mach = rng.uniform(0.5, 2.0, size=nbox)
    beta = np.exp(rng.uniform(math.log(0.3), math.log(3.0), size=nbox))
    return [dict(dims=tuple(int(x) for x in dims[b]), seed=1000 + b, mach=float(mach[b]),
                 beta=float(beta[b])) for b in range(nbox)]


def to_f32(state: torch.Tensor) -> torch.Tensor:
    """Round a float64 state to float32 (the GPU's storage precision)."""
    return state.to(torch.float32)


def as_oracle_input(state: torch.Tensor) -> np.ndarray:
    """float64 numpy copy (what the FP64 oracle consumes); rounding to float32
    first makes both paths start from the identical state."""
    return np.ascontiguousarray(state.to(torch.float32).to(torch.float64).cpu().numpy())
