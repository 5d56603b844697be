"""Scheme variants (ablations: minmod and superbee limiters, the exact fast
freezing speed, the per-pencil freezing speed) on the GPU against the FP64
oracle running the same
variant, with the tolerances of the default scheme's parity tests; the
default scheme is unaffected by switching back and forth."""
import numpy as np
import pytest
import torch

import oracle
from paper_1004_1680_gb300 import initial_conditions as ic
from tests.parity_util import G, field_scales, from_gpu, l1_rel, rel_err, to_gpu

pytestmark = pytest.mark.gpu
VARIANTS = [("minmod", "bound"), ("superbee", "bound"), ("vanleer", "fast"), ("vanleer", "pencil")]


@pytest.fixture(scope="module")
def mhd():
    from paper_1004_1680_gb300 import mhd as m
    m.load()
    return m


@pytest.fixture
def variant_oracle():
    yield oracle.set_scheme
    oracle.set_scheme("vanleer", "bound")


def box_of(mhd, st, lim, fr, xpath=0):
    nz, ny, nx = st.shape[1:]
    box = mhd.Box(nx, ny, nz, gamma=G)
    box.set_scheme(lim, fr)
    if xpath:
        box.set_xpath(xpath)
    box.set_state(to_gpu(st))
    return box


@pytest.mark.parametrize("lim,fr", VARIANTS)
@pytest.mark.parametrize("axis", [0, 1, 2])
@pytest.mark.parametrize("kind", [0, 1])
def test_variant_single_sweeps(mhd, variant_oracle, lim, fr, axis, kind):
    if kind == 1 and fr in ("fast", "pencil"):
        pytest.skip("the freezing speed does not enter the magnetic sweep")
    st = ic.turbulence((48, 40, 36), seed=21, dtype=torch.float64, kmin=1.0, kmax=4.0)
    s = ic.as_oracle_input(st)
    tau = 0.35 / oracle.cfl_rate(s, G)
    box = box_of(mhd, st, lim, fr)
    box.sweep(axis, kind, tau)
    g = from_gpu(box.get_state())
    variant_oracle(lim, fr)
    if kind == 0:
        oracle.fluid_sweep(s, axis, tau, G)
    else:
        oracle.mag_sweep(s, axis, tau)
    err = rel_err(g, s, field_scales(s))
    assert np.all(err < 1e-5), err
    box.close()


@pytest.mark.parametrize("lim,fr", VARIANTS)
@pytest.mark.parametrize("xpath", [1, 2])
def test_variant_steps(mhd, variant_oracle, lim, fr, xpath):
    st = ic.turbulence((32, 24, 20), seed=5, dtype=torch.float64, kmin=1.0, kmax=3.0)
    s = ic.as_oracle_input(st)
    S = field_scales(s)
    box = box_of(mhd, st, lim, fr, xpath)
    variant_oracle(lim, fr)
    t_orc, _ = oracle.run(s, 4, 0.7, G)
    box.run(4, 0.7)
    g = from_gpu(box.get_state())
    assert box.time() == pytest.approx(t_orc, rel=1e-5)
    assert np.all(rel_err(g, s, S) < 1e-4)
    assert np.all(l1_rel(g, s, S) < 1e-5)
    box.close()


def test_switching_back_restores_the_paper_scheme(mhd):
    st = ic.turbulence((32, 24, 20), seed=6, dtype=torch.float64, kmin=1.0, kmax=3.0)
    ref = box_of(mhd, st, "vanleer", "bound")
    ref.run(2, 0.7)
    box = box_of(mhd, st, "superbee", "bound")
    box.run(1, 0.7)
    box.set_scheme("vanleer", "bound")
    box.set_state(to_gpu(st))
    box.run(2, 0.7)
    assert torch.equal(box.get_state(), ref.get_state())
    with pytest.raises(RuntimeError):
        box.set_scheme("minmod", "fast")      # one ablation at a time
    box.close()
    ref.close()
