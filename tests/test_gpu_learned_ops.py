"""Kernels around the correction network against the oracle (oracle/ and
oracle/cnn.py): restriction, the conservative divergence-free projection and
its adjoint, the loss, the clipped application of a correction, and Adam."""
import numpy as np
import pytest
import torch

import oracle
from oracle import cnn
from paper_1004_1680_gb300 import initial_conditions as ic
from tests.parity_util import G

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mhd():
    from paper_1004_1680_gb300 import mhd as m
    m.load()
    return m


def div_b(s):
    n = s.shape[1:][::-1]
    d = np.zeros(s.shape[1:])
    for a in range(3):
        d += (np.roll(s[5 + a], -1, axis=2 - a) - s[5 + a]) * n[a]
    return d


def test_restriction_matches_oracle(mhd):
    st = ic.turbulence((32, 32, 32), seed=3, dtype=torch.float64, kmin=1.0, kmax=4.0)
    s32 = st.to(torch.float32)
    c = mhd.restrict(s32.contiguous().cuda(), 4).cpu().double().numpy()
    ref = oracle.restrict(s32.double().numpy().copy(), 4)
    assert np.max(np.abs(c - ref)) < 1e-6 * np.max(np.abs(ref))
    assert np.max(np.abs(div_b(c))) < 1e-4


def test_projection_against_oracle_and_adjoint(mhd):
    n = (16, 12, 8)
    cells = n[0] * n[1] * n[2]
    torch.manual_seed(0)
    y = torch.randn(cells, 8, device="cuda")
    scale = [1.0, 0.5, 0.5, 0.5, 2.0, 0.01]
    d = mhd.cnn_project(y, n, scale).cpu().double()
    y64 = y.cpu().double().T.reshape(8, n[2], n[1], n[0]).requires_grad_(True)
    dref = cnn.project(y64, scale)
    dr = dref.detach()
    for q in range(8):
        assert float((d[q] - dr[q]).abs().max()) < 1e-5 * float(dr[q].abs().max()), q
    dn = d.numpy()
    for q in range(5):
        assert abs(dn[q].sum()) < 1e-5 * np.abs(dn[q]).sum()
    assert np.max(np.abs(div_b(dn))) < 1e-5 * np.max(np.abs(dn[5:])) * 16
    # the backward kernel is the adjoint: against autograd of the oracle
    g = torch.randn(8, n[2], n[1], n[0], device="cuda")
    gy = mhd.cnn_project_backward(g, scale).float().cpu().double()   # (cells, 8)
    (dref * g.cpu().double()).sum().backward()
    gref = y64.grad.reshape(8, cells).T
    # BF16 output: each element within its rounding (2^-9 relative)
    assert bool(torch.all((gy - gref).abs() <= 2.0 ** -8 * gref.abs() + 1e-6 * gref.abs().max()))


def test_loss_and_gradient(mhd):
    torch.manual_seed(1)
    d = torch.randn(8, 8, 8, 8, device="cuda")
    t = torch.randn(8, 8, 8, 8, device="cuda")
    w = [0.1 * (q + 1) for q in range(8)]
    g = torch.empty_like(d)
    loss = mhd.cnn_loss(d, t, w, g=g)
    dn, tn = d.cpu().double().numpy(), t.cpu().double().numpy()
    ref = sum(w[q] * np.sum((dn[q] - tn[q]) ** 2) for q in range(8))
    assert float(loss.item()) == pytest.approx(ref, rel=1e-6)
    for q in range(8):
        assert np.allclose(g[q].cpu().numpy(), 2 * w[q] * (dn[q] - tn[q]), rtol=1e-5, atol=1e-6)


def test_correction_against_oracle(mhd):
    """Deliberately violent corrections: every branch of the clipping is taken.
    The oracle runs in FP32 so that both sides take each cell's decision in
    the kernel's precision; a cell may still decide differently where the
    thermal energy sits within rounding of its bound."""
    n = (16, 16, 16)
    st = ic.turbulence(n, seed=2, dtype=torch.float64, kmin=1.0, kmax=3.0).to(torch.float32)
    s = st.contiguous().cuda()
    div0 = np.max(np.abs(div_b(s.cpu().double().numpy())))
    torch.manual_seed(2)
    y = torch.randn(16 ** 3, 8, device="cuda") * 3.0
    d = mhd.cnn_project(y, n, [2.0, 2.0, 2.0, 2.0, 5.0, 0.05])
    ref, nref = cnn.correct(st, d.cpu())
    rho0 = s[0].clone()
    nclip = torch.zeros(1, dtype=torch.int32, device="cuda")
    mhd.correct(s, d, nclip=nclip)
    out = s.cpu()
    scale = ref.abs().amax(dim=(1, 2, 3))
    bad = torch.zeros(n[::-1], dtype=torch.bool)
    for q in range(8):
        bad |= (out[q] - ref[q]).abs() > 1e-5 * scale[q]
    assert int(bad.sum()) <= 2, int(bad.sum())
    eth0 = cnn.thermal_energy(st.double(), cnn.cell_magnetic_energy(st.double()))
    if bad.any():
        mag = cnn.cell_magnetic_energy(ref.double())
        margin = (cnn.thermal_energy(ref.double(), mag) - 0.5 * eth0).abs()
        assert torch.all(margin[bad] < 1e-4 * eth0[bad])
    assert abs(int(nclip.item()) - nref) <= 2 * int(bad.sum())
    assert nref > 0
    outn = out.double().numpy()
    assert np.all(outn[0] >= 0.5 * rho0.cpu().numpy() * (1 - 1e-6))
    assert np.min(oracle.pressure(outn, G)) > 0
    assert np.max(np.abs(div_b(outn))) < div0 + 1e-4 * np.max(np.abs(outn[5:])) * 16


def test_adam_against_oracle(mhd):
    torch.manual_seed(3)
    p = torch.randn(1000, device="cuda")
    m = torch.zeros_like(p)
    v = torch.zeros_like(p)
    pr = p.cpu().double()
    mr = torch.zeros_like(pr)
    vr = torch.zeros_like(pr)
    for step in range(1, 4):
        g = torch.randn(1000, device="cuda")
        mhd.adam(p, g, m, v, 1e-2, step)
        cnn.adam(pr, g.cpu().double(), mr, vr, 1e-2, step)
    assert torch.allclose(p.cpu().double(), pr, rtol=1e-5, atol=1e-6)


def test_network_entry_points_match_the_layer_calls():
    """mhd_cnn_forward / mhd_cnn_backward give the layer-by-layer results of
    the same kernels (forward bitwise; the gradients, whose block partials
    are added with atomics in any order, to FP32 rounding)."""
    from paper_1004_1680_gb300 import learned, mhd
    n = (16, 16, 4)
    cells = n[0] * n[1] * n[2]
    torch.manual_seed(5)
    net = learned.CorrectionNet(seed=3)
    for b in net.b:
        b.normal_(0.0, 0.1)
    x = (torch.randn(cells, 8, device="cuda") * 0.5).to(torch.bfloat16)
    y_ref, acts_ref = net.forward(x, n)
    acts = [torch.empty(cells, 32, dtype=torch.bfloat16, device="cuda") for _ in range(3)]
    y = torch.empty(cells, 8, device="cuda")
    mhd.cnn_forward(x, net.img, net.b, acts, y, n)
    torch.cuda.synchronize()
    assert torch.equal(y, y_ref)
    for a, r in zip(acts, acts_ref[1:]):
        assert torch.equal(a, r)
    gy = torch.randn(cells, 8, device="cuda").to(torch.bfloat16)
    net.backward(gy, acts_ref, n)
    gws = [torch.zeros_like(w) for w in net.W]
    gbs = [torch.zeros_like(b) for b in net.b]
    scratch = [torch.empty(cells, 32, dtype=torch.bfloat16, device="cuda") for _ in range(2)]
    mhd.cnn_backward(x, acts, gy, net.imgT, gws, gbs, scratch, n)
    torch.cuda.synchronize()
    L = len(net.W)
    for l in range(L):
        for got, want in ((gws[l], net.grads[l]), (gbs[l], net.grads[L + l])):
            scale = float(want.abs().max()) + 1e-30
            assert float((got - want).abs().max()) <= 1e-5 * scale
