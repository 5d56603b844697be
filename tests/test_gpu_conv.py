"""Tensor-core (tcgen05) periodic 3x3x3 convolution against PyTorch's FP64
CPU conv3d with circular padding, on BF16-rounded inputs and weights
(forward with bias and ReLU, input gradient through a ReLU mask, weight and
bias gradients)."""
import numpy as np
import pytest
import torch
import torch.nn.functional as F

pytestmark = pytest.mark.gpu


def to_ncdhw(x, n):
    nx, ny, nz = n
    return x.T.reshape(1, x.shape[1], nz, ny, nx)


def from_ncdhw(y):
    c = y.shape[1]
    return y.reshape(c, -1).T


@pytest.mark.parametrize("cin,cout", [(8, 32), (32, 32), (32, 8)])
def test_conv_forward_dgrad_wgrad(cin, cout):
    from paper_1004_1680_gb300 import mhd
    torch.manual_seed(cin * 100 + cout)
    n = (24, 32, 6)      # 3 x 2 x 6 tiles of 8 x 16 x 1, periodic wrap on every face
    cells = n[0] * n[1] * n[2]
    xb = (torch.randn(cells, cin) * 0.5).to(torch.bfloat16)
    w = torch.randn(cout, cin, 3, 3, 3) * 0.1
    wb = w.to(torch.bfloat16).float()
    bias = torch.randn(cout) * 0.1
    gyb = torch.randn(cells, cout).to(torch.bfloat16)
    # reference in FP64 on the CPU
    x64 = to_ncdhw(xb.double(), n).requires_grad_(True)
    w64 = wb.double().requires_grad_(True)
    b64 = bias.double().requires_grad_(True)
    z = F.conv3d(F.pad(x64, (1, 1, 1, 1, 1, 1), mode="circular"), w64, b64)
    z.backward(to_ncdhw(gyb.double(), n))
    zr = from_ncdhw(z.detach())
    # GPU
    dev = "cuda"
    xg, gyg = xb.to(dev), gyb.to(dev)
    img = mhd.conv_pack(w.to(dev))
    _, y32 = mhd.conv3d(xg, img, n, cin, cout, bias=bias.to(dev), out_bf16=False, out_f32=True)
    _, yr = mhd.conv3d(xg, img, n, cin, cout, bias=bias.to(dev), relu=True, out_bf16=False, out_f32=True)
    imgt = mhd.conv_pack(w.to(dev), transpose=True)
    _, gx = mhd.conv3d(gyg, imgt, n, cout, cin, flip=True, out_bf16=False, out_f32=True)
    mask = xb.to(dev)
    _, gxm = mhd.conv3d(gyg, imgt, n, cout, cin, flip=True, mask=mask, out_bf16=False, out_f32=True)
    gw = torch.zeros(cout * cin * 27, device=dev)
    gb = torch.zeros(cout, device=dev)
    mhd.conv3d_wgrad(xg, gyg, n, cin, cout, gw, gb)
    torch.cuda.synchronize()
    assert mhd.conv_error() == 0
    scale = float(zr.abs().max())
    assert float((y32.cpu().double() - zr).abs().max()) < 1e-4 * scale
    assert torch.equal(yr.cpu(), torch.clamp(y32.cpu(), min=0.0))
    gxr = from_ncdhw(x64.grad)
    assert float((gx.cpu().double() - gxr).abs().max()) < 1e-4 * float(gxr.abs().max())
    gxmr = torch.where(xb.double() > 0, gxr, torch.zeros_like(gxr))
    assert float((gxm.cpu().double() - gxmr).abs().max()) < 1e-4 * float(gxr.abs().max())
    gwr = w64.grad.reshape(-1)
    assert float((gw.cpu().double() - gwr).abs().max()) < 1e-4 * float(gwr.abs().max())
    assert float((gb.cpu().double() - b64.grad).abs().max()) < 1e-4 * float(b64.grad.abs().max())


@pytest.mark.parametrize("n", [(12, 8, 4), (8, 16, 2)])
def test_wgrad_paths(n):
    """Weight and bias gradient of a box that does not tile into 8 x 16 x 1
    cells (CUDA-core path) and of a single-tile-row box (tensor-core path,
    every tap's halo wraps), against FP64 autograd."""
    from paper_1004_1680_gb300 import mhd
    torch.manual_seed(7)
    cin, cout = 32, 8
    cells = n[0] * n[1] * n[2]
    xb = (torch.randn(cells, cin) * 0.5).to(torch.bfloat16)
    gyb = torch.randn(cells, cout).to(torch.bfloat16)
    x64 = to_ncdhw(xb.double(), n)
    w64 = torch.zeros(cout, cin, 3, 3, 3, dtype=torch.float64, requires_grad=True)
    b64 = torch.zeros(cout, dtype=torch.float64, requires_grad=True)
    F.conv3d(F.pad(x64, (1, 1, 1, 1, 1, 1), mode="circular"), w64, b64).backward(to_ncdhw(gyb.double(), n))
    gw = torch.zeros(cout * cin * 27, device="cuda")
    gb = torch.zeros(cout, device="cuda")
    mhd.conv3d_wgrad(xb.cuda(), gyb.cuda(), n, cin, cout, gw, gb)
    torch.cuda.synchronize()
    assert mhd.conv_error() == 0
    gwr = w64.grad.reshape(-1)
    assert float((gw.cpu().double() - gwr).abs().max()) < 1e-4 * float(gwr.abs().max())
    assert float((gb.cpu().double() - b64.grad).abs().max()) < 1e-4 * float(b64.grad.abs().max())


def sampled_conv(x, w, n, cells, flip=False):
    """FP64 output of the circular cross-correlation at the given cells only:
    y[c, o] = sum_{ci, taps} w[o, ci, tap] x[c + s * offset(tap), ci]."""
    nx, ny, nz = n
    i, j, k = cells % nx, (cells // nx) % ny, cells // (nx * ny)
    s = -1 if flip else 1
    out = np.zeros((len(cells), w.shape[0]))
    for kz in range(3):
        for ky in range(3):
            for kx in range(3):
                src = ((i + s * (kx - 1)) % nx) + nx * (((j + s * (ky - 1)) % ny) + ny * ((k + s * (kz - 1)) % nz))
                out += x[src] @ w[:, :, kz, ky, kx].T
    return out


@pytest.mark.parametrize("cin,cout", [(8, 32), (32, 32), (32, 8)])
def test_conv_64_cubed_sampled(cin, cout):
    """The 64^3 configuration the correction runs on (2048 tiles: every block
    loops over several tiles with the next halo prefetched), forward and
    input gradient, at 4096 sampled cells computed one by one in FP64."""
    from paper_1004_1680_gb300 import mhd
    n = (64, 64, 64)
    N = n[0] * n[1] * n[2]
    g = torch.Generator().manual_seed(cin + 7 * cout)
    xb = (torch.randn(N, cin, generator=g) * 0.5).to(torch.bfloat16)
    gyb = torch.randn(N, cout, generator=g).to(torch.bfloat16)
    w = torch.randn(cout, cin, 3, 3, 3, generator=g) * 0.1
    bias = torch.randn(cout, generator=g) * 0.1
    img = mhd.conv_pack(w.cuda())
    imgt = mhd.conv_pack(w.cuda(), transpose=True)
    _, y = mhd.conv3d(xb.cuda(), img, n, cin, cout, bias=bias.cuda(), out_bf16=False, out_f32=True)
    _, gx = mhd.conv3d(gyb.cuda(), imgt, n, cout, cin, flip=True, out_bf16=False, out_f32=True)
    torch.cuda.synchronize()
    assert mhd.conv_error() == 0
    rng = np.random.default_rng(cin * cout)
    cells = np.concatenate([rng.integers(0, N, 4000), [0, N - 1, 63, 64 * 64 - 1, N - 64 * 64]])
    wb = w.to(torch.bfloat16).double().numpy()
    ref = sampled_conv(xb.double().numpy(), wb, n, cells) + bias.double().numpy()
    assert np.max(np.abs(y.cpu().double().numpy()[cells] - ref)) < 1e-4 * np.max(np.abs(ref))
    wt = np.transpose(wb, (1, 0, 2, 3, 4))          # input gradient: transposed, mirrored taps
    refg = sampled_conv(gyb.double().numpy(), wt, n, cells, flip=True)
    assert np.max(np.abs(gx.cpu().double().numpy()[cells] - refg)) < 1e-4 * np.max(np.abs(refg))
    # every cell written (no tile skipped): finite everywhere
    assert bool(torch.isfinite(y).all()) and bool(torch.isfinite(gx).all())
