"""The correction network trained with the project's own kernels: forward
output and every weight/bias gradient of the full training graph (network,
conservative divergence-free projection, weighted MSE) against PyTorch FP64
autograd of the same graph (circular conv3d as the library oracle), with the
same BF16 rounding of weights and activations."""
import numpy as np
import pytest
import torch
import torch.nn.functional as F

from paper_1004_1680_gb300 import initial_conditions as ic

pytestmark = pytest.mark.gpu


def torch_pipeline(x_cells, W, b, n, scale, weight, target):
    """FP64 reference of forward + projection + loss; x_cells (cells, 8)."""
    nx, ny, nz = n
    h = x_cells.T.reshape(1, 8, nz, ny, nx)
    L = len(W)
    for li in range(L):
        z = F.conv3d(F.pad(h, (1, 1, 1, 1, 1, 1), mode="circular"), W[li], b[li])
        if li < L - 1:
            h = torch.relu(z).to(torch.bfloat16).to(torch.float64)   # BF16 activations as on the GPU
        else:
            h = z
    y = h[0]                                                       # (8, nz, ny, nx)
    d = [scale[q] * y[q] for q in range(5)]
    d = [dq - dq.mean() for dq in d]
    A = [scale[5] * y[5 + c] for c in range(3)]
    up = lambda a, ax: torch.roll(a, shifts=-1, dims=ax)         # +1 along numpy axis
    bx = (up(A[2], 1) - A[2]) * ny - (up(A[1], 0) - A[1]) * nz
    by = (up(A[0], 0) - A[0]) * nz - (up(A[2], 2) - A[2]) * nx
    bz = (up(A[1], 2) - A[1]) * nx - (up(A[0], 1) - A[0]) * ny
    d = torch.stack(d + [bx, by, bz])
    loss = sum(weight[q] * ((d[q] - target[q]) ** 2).sum() for q in range(8))
    return y, d, loss


def test_training_graph_against_fp64_autograd():
    from paper_1004_1680_gb300 import learned, mhd
    n = (16, 8, 8)
    cells = n[0] * n[1] * n[2]
    st = ic.turbulence(n, seed=4, dtype=torch.float64, kmin=1.0, kmax=2.0).to(torch.float32).contiguous().cuda()
    torch.manual_seed(5)
    target = (torch.randn(8, n[2], n[1], n[0]) * 0.01).cuda()
    norm = learned.Norm(mu=[float(st[q].mean()) for q in range(8)],
                        inv_sigma=[1.0 / max(float(st[q].std()), 1e-3) for q in range(8)],
                        out_scale=[0.01, 0.02, 0.02, 0.02, 0.05, 0.001],
                        loss_weight=[1.0 / cells] * 8)
    net = learned.CorrectionNet(seed=1, out_scale=1.0)
    corr = learned.Corrector(net, norm, n)
    # GPU forward + backward
    mhd.cnn_normalize(st, norm.mu, norm.inv_sigma, out=corr.x)
    y, acts = net.forward(corr.x, n)
    d = mhd.cnn_project(y, n, norm.out_scale, out=corr.d, sums=corr.sums)
    g = torch.empty_like(d)
    loss = mhd.cnn_loss(d, target, norm.loss_weight, g=g)
    gy = mhd.cnn_project_backward(g, norm.out_scale)
    net.backward(gy, acts, n)
    torch.cuda.synchronize()
    assert mhd.conv_error() == 0
    # FP64 reference on the CPU with the GPU's BF16 input and BF16-rounded weights
    x64 = corr.x.cpu().double()
    W = [w.to(torch.bfloat16).double().cpu().requires_grad_(True) for w in net.W]
    b = [bb.double().cpu().requires_grad_(True) for bb in net.b]
    yr, dr, lr = torch_pipeline(x64, W, b, n, norm.out_scale, norm.loss_weight, target.cpu().double())
    lr.backward()
    yg = y.cpu().double().T.reshape(8, n[2], n[1], n[0])
    assert float((yg - yr.detach()).abs().max()) < 2e-2 * float(yr.abs().max())
    assert float(loss.item()) == pytest.approx(float(lr.item()), rel=5e-2)
    for li in range(len(W)):
        gw, gwr = net.grads[li].cpu().double(), W[li].grad
        assert float((gw - gwr).abs().max()) < 5e-2 * float(gwr.abs().max()), li
        gb, gbr = net.grads[len(W) + li].cpu().double(), b[li].grad
        assert float((gb - gbr).abs().max()) < 5e-2 * float(gbr.abs().max()) + 1e-12, li


def test_training_reduces_loss_on_solver_pairs():
    """A few epochs on pairs made by the solver itself (small grids)."""
    from paper_1004_1680_gb300 import learned
    inputs, targets = learned.generate_pairs([7], steps_per_seed=6, nf=64, r=4)
    norm = learned.make_norm(inputs, targets, inputs.shape[-1])
    net, hist = learned.train(inputs, targets, norm, epochs=6, lr=2e-3)
    assert hist[-1] < hist[0]
