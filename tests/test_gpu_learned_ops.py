"""Kernels around the correction network: restriction (against the oracle),
the conservative divergence-free projection and its adjoint, the loss, the
clipped application of a correction, and Adam."""
import numpy as np
import pytest
import torch

import oracle
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


def test_projection_is_conservative_divergence_free_and_adjoint(mhd):
    n = (16, 16, 16)
    cells = 16 ** 3
    torch.manual_seed(0)
    y = torch.randn(cells, 8, device="cuda")
    scale = [1.0, 0.5, 0.5, 0.5, 2.0, 0.01]
    d = mhd.cnn_project(y, n, scale).cpu().double().numpy()
    for q in range(5):
        assert abs(d[q].sum()) < 1e-5 * np.abs(d[q]).sum()
    assert np.max(np.abs(div_b(d))) < 1e-5 * np.max(np.abs(d[5:])) * 16
    g = torch.randn(8, 16, 16, 16, device="cuda")
    gy = mhd.cnn_project_backward(g, scale).float().cpu().double().numpy()
    lhs = float(np.sum(d * g.cpu().double().numpy()))
    rhs = float(np.sum(y.cpu().double().numpy() * gy))
    assert abs(lhs - rhs) < 2e-2 * np.linalg.norm(y.cpu().numpy()) * np.linalg.norm(gy)


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


def test_correction_keeps_state_physical(mhd):
    st = ic.turbulence((16, 16, 16), seed=2, dtype=torch.float64, kmin=1.0, kmax=3.0).to(torch.float32)
    s = st.contiguous().cuda()
    div0 = np.max(np.abs(div_b(s.cpu().double().numpy())))
    torch.manual_seed(2)
    y = torch.randn(16 ** 3, 8, device="cuda") * 3.0
    d = mhd.cnn_project(y, (16, 16, 16), [2.0, 2.0, 2.0, 2.0, 5.0, 0.05])   # deliberately violent
    rho0 = s[0].clone()
    nclip = torch.zeros(1, dtype=torch.int32, device="cuda")
    mhd.correct(s, d, nclip=nclip)
    out = s.cpu().double().numpy()
    assert np.all(out[0] >= 0.5 * rho0.cpu().numpy() * (1 - 1e-6))
    assert np.min(oracle.pressure(out, G)) > 0
    assert np.max(np.abs(div_b(out))) < div0 + 1e-4 * np.max(np.abs(out[5:])) * 16
    assert int(nclip.item()) > 0


def test_adam_matches_formula(mhd):
    torch.manual_seed(3)
    p = torch.randn(1000, device="cuda")
    m = torch.zeros_like(p)
    v = torch.zeros_like(p)
    pr = p.cpu().double().numpy().copy()
    mr = np.zeros_like(pr)
    vr = np.zeros_like(pr)
    for step in range(1, 4):
        g = torch.randn(1000, device="cuda")
        mhd.adam(p, g, m, v, 1e-2, step)
        gn = g.cpu().double().numpy()
        mr = 0.9 * mr + 0.1 * gn
        vr = 0.999 * vr + 0.001 * gn * gn
        pr -= 1e-2 * (mr / (1 - 0.9 ** step)) / (np.sqrt(vr / (1 - 0.999 ** step)) + 1e-8)
    assert np.allclose(p.cpu().numpy(), pr, rtol=1e-5, atol=1e-6)
