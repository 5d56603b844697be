"""Pins of the learned-correction oracle (oracle/cnn.py) to what fixes it
independently of itself: brute-force convolution, closed-form discrete curls
of single Fourier modes, exact conservation and solenoidality, central finite
differences of the training graph, the invariants of the clipped correction,
and Adam's closed form under a constant gradient."""
import itertools
import math

import numpy as np
import pytest
import torch

from oracle import cnn
from paper_1004_1680_gb300 import initial_conditions as ic
from tests.parity_util import G


@pytest.fixture(autouse=True)
def _fp64_default():
    old = torch.get_default_dtype()
    torch.set_default_dtype(torch.float64)
    yield
    torch.set_default_dtype(old)


def test_conv3d_circular_against_brute_force():
    g = torch.Generator().manual_seed(0)
    cin, cout, n = 2, 3, (5, 4, 3)              # (nx, ny, nz)
    h = torch.randn(1, cin, n[2], n[1], n[0], generator=g)
    w = torch.randn(cout, cin, 3, 3, 3, generator=g)
    b = torch.randn(cout, generator=g)
    out = cnn.conv3d_circular(h, w, b)[0].numpy()
    hn, wn = h[0].numpy(), w.numpy()
    ref = np.zeros_like(out)
    for o, z, y, x in itertools.product(range(cout), range(n[2]), range(n[1]), range(n[0])):
        acc = b[o].item()
        for c, dz, dy, dx in itertools.product(range(cin), range(3), range(3), range(3)):
            acc += wn[o, c, dz, dy, dx] * hn[c, (z + dz - 1) % n[2], (y + dy - 1) % n[1], (x + dx - 1) % n[0]]
        ref[o, z, y, x] = acc
    assert np.max(np.abs(out - ref)) < 1e-12


@pytest.mark.parametrize("c,e", [(c, e) for c in range(3) for e in range(3) if c != e])
def test_curl_of_single_mode_closed_form(c, e):
    """A_c = cos(2 pi k x_e) on its edges gives b_f = eps_{f e c} dA_c/dx_e with
    the centred difference of a cosine: -2 sin(2 pi k x) sin(pi k h) / h at the
    face positions (cell-centred along e)."""
    n = [12, 10, 8]                             # nx, ny, nz
    f = 3 - c - e
    k = 2
    A = [torch.zeros(n[2], n[1], n[0]) for _ in range(3)]
    idx = torch.arange(n[e], dtype=torch.float64)
    h = 1.0 / n[e]
    shape = [1, 1, 1]
    shape[2 - e] = n[e]
    A[c] = torch.cos(2 * math.pi * k * idx * h).reshape(shape).expand(n[2], n[1], n[0]).clone()  # edges at i h
    b = cnn.curl_edges(A)
    xc = (idx + 0.5) * h
    deriv = (-2.0 * torch.sin(2 * math.pi * k * xc) * math.sin(math.pi * k * h) / h).reshape(shape)
    perm_sign = {(0, 1, 2): 1, (1, 2, 0): 1, (2, 0, 1): 1, (0, 2, 1): -1, (2, 1, 0): -1, (1, 0, 2): -1}[(f, e, c)]
    assert torch.max(torch.abs(b[f] - perm_sign * deriv)) < 1e-12 * n[e]
    for other in range(3):
        if other != f:
            assert torch.max(torch.abs(b[other])) == 0.0


def test_projection_conserves_and_keeps_div_b():
    g = torch.Generator().manual_seed(1)
    y = torch.randn(8, 6, 10, 8, generator=g)
    scale = [0.3, 0.1, 0.2, 0.4, 1.5, 0.02]
    d = cnn.project(y, scale)
    for q in range(5):
        assert abs(float(d[q].sum())) < 1e-12 * float(d[q].abs().sum())
        # a constant shift of the scaled output, nothing else
        diff = d[q] - scale[q] * y[q]
        assert float(diff.max() - diff.min()) < 1e-13
    assert float(cnn.divergence(list(d[5:8])).abs().max()) < 1e-12 * float(d[5:8].abs().max()) * 10
    # a constant potential has no curl; the face totals of a curl vanish
    assert float(cnn.curl_edges([torch.ones(6, 10, 8)] * 3)[0].abs().max()) == 0.0
    for q in range(5, 8):
        assert abs(float(d[q].sum())) < 1e-12 * float(d[q].abs().sum())


def test_divergence_of_turbulence_initial_field():
    st = ic.turbulence((16, 16, 16), seed=2, dtype=torch.float64, kmin=1.0, kmax=3.0)
    assert float(cnn.divergence(list(st[5:8])).abs().max()) < 1e-12 * 16


def test_training_graph_gradient_by_central_differences():
    torch.manual_seed(2)
    n = (4, 4, 4)
    W = [torch.randn(co, ci, 3, 3, 3) * (1.0 / math.sqrt(27 * ci)) for ci, co in cnn.LAYERS]
    b = [torch.randn(co) * 0.1 for _, co in cnn.LAYERS]
    for t in W + b:
        t.requires_grad_(True)
    x = torch.randn(8, n[2], n[1], n[0])
    target = torch.randn(8, n[2], n[1], n[0]) * 0.1
    scale = [0.1, 0.2, 0.2, 0.2, 0.3, 0.05]
    weight = [1.0 + q for q in range(8)]
    _, _, L = cnn.training_graph(x, W, b, scale, weight, target)
    L.backward()
    eps = 1e-6
    gen = torch.Generator().manual_seed(3)
    for li in range(len(W)):
        for param in (W[li], b[li]):
            flat = param.detach().view(-1)
            for j in torch.randint(0, flat.numel(), (4,), generator=gen).tolist():
                with torch.no_grad():
                    old = flat[j].item()
                    flat[j] = old + eps
                    lp = cnn.training_graph(x, W, b, scale, weight, target)[2].item()
                    flat[j] = old - eps
                    lm = cnn.training_graph(x, W, b, scale, weight, target)[2].item()
                    flat[j] = old
                fd = (lp - lm) / (2 * eps)
                ad = param.grad.view(-1)[j].item()
                assert abs(fd - ad) < 1e-5 * max(1.0, abs(ad)), (li, j, fd, ad)


def _state():
    return ic.turbulence((8, 8, 8), seed=5, dtype=torch.float64, kmin=1.0, kmax=2.0)


def test_zero_and_small_corrections_are_applied_exactly():
    s = _state()
    out, nclip = cnn.correct(s, torch.zeros_like(s))
    assert torch.equal(out, s) and nclip == 0
    g = torch.Generator().manual_seed(4)
    d = cnn.project(torch.randn(8, 8, 8, 8, generator=g), [1e-4, 1e-4, 1e-4, 1e-4, 1e-4, 1e-6])
    out, nclip = cnn.correct(s, d)
    assert nclip == 0
    assert torch.equal(out, s + d)


def test_violent_correction_invariants():
    s = _state()
    g = torch.Generator().manual_seed(5)
    d = cnn.project(3.0 * torch.randn(8, 8, 8, 8, generator=g), [2.0, 2.0, 2.0, 2.0, 5.0, 0.05])
    out, nclip = cnn.correct(s, d)
    assert nclip > 0
    eth0 = cnn.thermal_energy(s, cnn.cell_magnetic_energy(s))
    mag = cnn.cell_magnetic_energy(out)
    eth = cnn.thermal_energy(out, mag)
    assert torch.all(out[0] >= 0.5 * s[0] * (1 - 1e-15))
    assert torch.all(eth >= 0.5 * eth0 * (1 - 1e-12))
    assert torch.equal(out[5:8], s[5:8] + d[5:8])
    div0 = cnn.divergence(list(s[5:8])).abs().max()
    assert float(cnn.divergence(list(out[5:8])).abs().max()) < float(div0) + 1e-11
    # maximality: where a cell took a < 1, the next larger a violates the bound
    du = d[0:5].clone()
    du[0] = torch.maximum(d[0], -0.5 * s[0])
    a = torch.full_like(s[0], -1.0)
    for cand in (1.0, 0.5, 0.25, 0.0):
        hit = torch.all(torch.isclose(out[0:5], s[0:5] + cand * du, rtol=0, atol=1e-14), dim=0) & (a < 0)
        a = torch.where(hit, torch.full_like(a, cand), a)
    raised = a < 0
    assert torch.all(torch.isclose(eth[raised], 0.5 * eth0[raised], rtol=1e-12))
    for cand, larger in ((0.5, 1.0), (0.25, 0.5), (0.0, 0.25)):
        sel = a == cand
        if sel.any():
            u = s[0:5] + larger * du
            e_try = u[4] - 0.5 * (u[1] ** 2 + u[2] ** 2 + u[3] ** 2) / u[0] - mag
            assert torch.all(e_try[sel] < 0.5 * eth0[sel])
    p = (G - 1) * eth
    assert torch.all(p > 0)


def test_adam_closed_form_for_constant_gradient():
    """With a constant gradient g, both bias-corrected moments are exact
    (m_hat = g, v_hat = g^2) at every step, so each step moves p by
    lr g / (|g| + eps)."""
    g = torch.tensor([0.3, -2.0, 1e-3, 0.0])
    p = torch.tensor([1.0, 2.0, 3.0, 4.0])
    p0 = p.clone()
    m, v = torch.zeros(4), torch.zeros(4)
    for t in range(1, 8):
        cnn.adam(p, g, m, v, 1e-2, t)
        expect = p0 - t * 1e-2 * g / (g.abs() + 1e-8)
        assert torch.allclose(p, expect, rtol=0, atol=1e-12)
