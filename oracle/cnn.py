"""FP64 CPU oracle of the learned coarse-grid correction (test infrastructure).

Only the test suite may import this module.  The method has no counterpart in
the paper (whose solver has no learned part); what it computes is defined
here from plain definitions, with PyTorch CPU operations as library
primitives:

* ``network``: four 3x3x3 convolutions with circular (periodic) padding,
  8 -> 32 -> 32 -> 32 -> 8 channels, ReLU between layers.
* ``project``: the network output y (8 channels) read as five cell
  corrections scaled by s_q, each with its box mean removed (so the totals of
  rho, m and e are unchanged), and three edge vector potentials A = s_A y_5..7
  whose discrete curl is the face-field correction (so the discrete
  divergence of b, the one of Eq. 5, is unchanged).
* ``loss``: sum_q w_q sum_cells (d_q - t_q)^2.
* ``correct``: the clipped application of a correction to a state.
* ``adam``: the bias-corrected Adam step (Kingma & Ba 2015, Algorithm 1).

Arrays are float64 torch tensors of shape (8, nz, ny, nx) unless stated;
b_d[k, j, i] lives on the low face of cell (i, j, k) along d; the edge
potential A_x lives on the x-edge (i, j-1/2, k-1/2), A_y on (i-1/2, j, k-1/2),
A_z on (i-1/2, j-1/2, k).  Periodic unit box, h_d = 1/n_d.
"""
from __future__ import annotations

import torch
import torch.nn.functional as F

LAYERS = [(8, 32), (32, 32), (32, 32), (32, 8)]


def conv3d_circular(h: torch.Tensor, w: torch.Tensor, b: torch.Tensor | None) -> torch.Tensor:
    """3x3x3 cross-correlation with periodic wrap: h (1, cin, nz, ny, nx),
    w (cout, cin, 3, 3, 3); out[o, z, y, x] = b[o] + sum w[o, c, dz, dy, dx]
    h[c, z+dz-1, y+dy-1, x+dx-1] (indices mod n)."""
    return F.conv3d(F.pad(h, (1, 1, 1, 1, 1, 1), mode="circular"), w, b)


def network(x: torch.Tensor, W, b, act_round=None) -> torch.Tensor:
    """x (8, nz, ny, nx) -> y (8, nz, ny, nx); act_round (e.g. a BF16 round
    trip) is applied to the hidden activations after the ReLU."""
    h = x.unsqueeze(0)
    for li in range(len(W)):
        h = conv3d_circular(h, W[li], b[li])
        if li < len(W) - 1:
            h = torch.relu(h)
            if act_round is not None:
                h = act_round(h)
    return h[0]


def _up(a: torch.Tensor, axis: int) -> torch.Tensor:
    """a at index + 1 along array axis (periodic)."""
    return torch.roll(a, shifts=-1, dims=axis)


def curl_edges(A) -> list:
    """Face field b = curl A of edge potentials (A_x, A_y, A_z), each (nz, ny, nx).

    b_x at face (i-1/2, j, k) = dA_z/dy - dA_y/dz with the differences taken
    between the edges bounding that face; likewise for b_y and b_z.
    """
    nz, ny, nx = A[0].shape
    bx = (_up(A[2], 1) - A[2]) * ny - (_up(A[1], 0) - A[1]) * nz
    by = (_up(A[0], 0) - A[0]) * nz - (_up(A[2], 2) - A[2]) * nx
    bz = (_up(A[1], 2) - A[1]) * nx - (_up(A[0], 1) - A[0]) * ny
    return [bx, by, bz]


def divergence(bf) -> torch.Tensor:
    """Discrete divergence of a face field (b_x, b_y, b_z) per cell (Eq. 5)."""
    nz, ny, nx = bf[0].shape
    return ((_up(bf[0], 2) - bf[0]) * nx + (_up(bf[1], 1) - bf[1]) * ny + (_up(bf[2], 0) - bf[2]) * nz)


def project(y: torch.Tensor, scale) -> torch.Tensor:
    """Correction d (8, nz, ny, nx) from the network output y: d_q = s_q y_q
    minus its box mean for q < 5; (d_5, d_6, d_7) = curl of A = s_A y_5..7.
    scale = (s_rho, s_mx, s_my, s_mz, s_e, s_A)."""
    d = [scale[q] * y[q] for q in range(5)]
    d = [dq - dq.mean() for dq in d]
    A = [scale[5] * y[5 + c] for c in range(3)]
    return torch.stack(d + curl_edges(A))


def loss(d: torch.Tensor, target: torch.Tensor, weight) -> torch.Tensor:
    return sum(weight[q] * ((d[q] - target[q]) ** 2).sum() for q in range(8))


def training_graph(x: torch.Tensor, W, b, scale, weight, target, act_round=None):
    """(y, d, loss) of one training sample; gradients by autograd."""
    y = network(x, W, b, act_round)
    d = project(y, scale)
    return y, d, loss(d, target, weight)


def cell_magnetic_energy(s: torch.Tensor) -> torch.Tensor:
    """|b_c|^2 / 2 with b_c the mean of each cell's two faces."""
    bx = 0.5 * (s[5] + _up(s[5], 2))
    by = 0.5 * (s[6] + _up(s[6], 1))
    bz = 0.5 * (s[7] + _up(s[7], 0))
    return 0.5 * (bx * bx + by * by + bz * bz)


def thermal_energy(s: torch.Tensor, mag: torch.Tensor) -> torch.Tensor:
    """e - |m|^2 / (2 rho) - |b_c|^2 / 2 (p / (gamma - 1) by Eq. 3)."""
    return s[4] - 0.5 * (s[1] * s[1] + s[2] * s[2] + s[3] * s[3]) / s[0] - mag


def correct(s: torch.Tensor, d: torch.Tensor):
    """Apply correction d to state s (returns (new state, clipped-cell count)).

    1. Faces: b += d_b, unscaled (keeps the divergence unchanged).
    2. Per cell: the density correction is clipped at -rho/2; the cell
       correction (rho, m, e) is then scaled by the largest a in
       {1, 1/2, 1/4, 0} that keeps the thermal energy, evaluated with the
       corrected faces, at or above half its value in the uncorrected state;
       if no a does, the uncorrected cell is kept with e raised to that bound.
    The count adds one per cell for a clipped density, for a < 1, and for
    the raised energy.  Evaluated in the dtype of s.
    """
    eth0 = thermal_energy(s, cell_magnetic_energy(s))
    out = s.clone()
    out[5:8] = s[5:8] + d[5:8]
    mag = cell_magnetic_energy(out)
    floor_e = 0.5 * eth0
    du = d[0:5].clone()
    du[0] = torch.maximum(d[0], -0.5 * s[0])
    nclip = int((du[0] != d[0]).sum())
    chosen = torch.zeros_like(s[0], dtype=torch.bool)
    cells = s[0:5].clone()
    for a in (1.0, 0.5, 0.25, 0.0):
        u = s[0:5] + a * du
        ok = (u[4] - 0.5 * (u[1] * u[1] + u[2] * u[2] + u[3] * u[3]) / u[0] - mag >= floor_e) & ~chosen
        cells = torch.where(ok.unsqueeze(0), u, cells)
        nclip += int(ok.sum()) if a < 1.0 else 0
        chosen |= ok
    raise_e = ~chosen
    kin = 0.5 * (s[1] * s[1] + s[2] * s[2] + s[3] * s[3]) / s[0]
    cells[4] = torch.where(raise_e, kin + mag + floor_e, cells[4])
    nclip += int(raise_e.sum())
    out[0:5] = cells
    return out, nclip


def adam(p, g, m, v, lr: float, step: int, b1: float = 0.9, b2: float = 0.999, eps: float = 1e-8):
    """One Adam step in place on p, m, v (step counts from 1)."""
    m.mul_(b1).add_((1 - b1) * g)
    v.mul_(b2).add_((1 - b2) * g * g)
    mhat = m / (1 - b1 ** step)
    vhat = v / (1 - b2 ** step)
    p.sub_(lr * mhat / (vhat.sqrt() + eps))
