"""TMA-staged sweeps (kernel axes 1 and 2) against the register-load sweeps
and against the FP64 oracle.

A staged sweep reads the same values and does the same arithmetic as the
register-load sweep, except that the staged fluid sweep takes the freezing
speeds' square roots from the hardware approximation (a few ulp): magnetic
sweeps must be bitwise those of the register path, and fluid sweeps and
full steps equal to it within FP32 rounding (1e-6 of the field scales, four
orders below the one-step parity bound against the oracle).  Covered: single
fluid and magnetic sweeps, full steps with the fused CFL rate and the fused
pair of z magnetic sweeps, the optional pressure floor, segmented pencils
(interior segments never cross the periodic wrap, the end segments do) and
the x sweeps through the exchanged layout (kernel axis 1 with the lanes
along y).  A fluid sweep qualifies when its rows are a multiple of 16 bytes
(tiles cut by the box's end included); a magnetic sweep when the contiguous
axis is a multiple of 32 and the row axis a multiple of 8; `tma_sweeps`
shows that the staged kernels ran.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1004_1680_gb300 import initial_conditions as ic
from tests.parity_util import G, field_scales, from_gpu, rel_err, to_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mhd():
    from paper_1004_1680_gb300 import mhd as m
    m.load()
    return m


def pair(mhd, st64, **cfg):
    nz, ny, nx = st64.shape[1:]
    boxes = []
    for tma in (True, False):
        b = mhd.Box(nx, ny, nz, gamma=G)
        b.set_tma(tma)
        if "segs" in cfg:
            b.set_segments(*cfg["segs"])
        if "xpath" in cfg:
            b.set_xpath(cfg["xpath"])
        if "floor" in cfg:
            b.set_pressure_floor(cfg["floor"])
        b.set_state(to_gpu(st64))
        boxes.append(b)
    return boxes


def close_to(a, b, tol=1e-6):
    """max per-field |a - b| / field scale, the scales of the FP64 state a"""
    sa = a.to(torch.float64).cpu().numpy()
    err = rel_err(b.to(torch.float64).cpu().numpy(), sa, field_scales(sa))
    return bool(np.all(err < tol)), err


@pytest.mark.parametrize("axis", [1, 2])
@pytest.mark.parametrize("kind", [0, 1])
def test_single_staged_sweep_matches_the_register_sweep(mhd, axis, kind):
    st = ic.turbulence((64, 32, 24), seed=31, dtype=torch.float64, kmin=1.0, kmax=4.0)
    a, b = pair(mhd, st)
    tau = 0.35 / oracle.cfl_rate(ic.as_oracle_input(st), G)
    a.sweep(axis, kind, tau)
    b.sweep(axis, kind, tau)
    assert a.tma_sweeps() == 1 and b.tma_sweeps() == 0
    if kind == 1:  # the magnetic sweeps share all of their arithmetic
        assert torch.equal(a.get_state(), b.get_state())
    else:
        ok, err = close_to(a.get_state(), b.get_state())
        assert ok, err


@pytest.mark.parametrize("dims, cfg", [
    ((32, 32, 32), {}),                                  # one block column, whole pencils
    ((64, 32, 24), {"segs": (0, 16, 4)}),                # z segments of 4: wrapped chunks in every segment
    ((32, 64, 48), {"segs": (0, 32, 16)}),               # interior segments with no wrap
    ((64, 64, 16), {"xpath": 2}),                        # x sweeps through the exchanged layout
    ((32, 32, 24), {"floor": 1e-3}),                     # the pressure-floor variant
    ((96, 32, 28), {"segs": (0, 8, 0), "xpath": 2}),     # 3 block columns, ragged z chunking
    ((32, 16, 16), {}),                                  # the shortest staged pencils (16), rows of 16
    ((32, 8, 16), {"segs": (0, 0, 4)}),                  # rows of 8 (z sweeps staged, y pencils too short)
    ((44, 36, 22), {}),                                  # fluid tiles cut by the box's end (lanes 12, rows 2)
    ((52, 24, 30), {"xpath": 2, "segs": (0, 8, 0)}),     # ragged lanes along y on the exchanged layout too
])
def test_staged_steps_match_the_register_steps(mhd, dims, cfg):
    st = ic.turbulence(dims, seed=37, dtype=torch.float64, kmin=1.0, kmax=3.0, mach=0.8)
    a, b = pair(mhd, st, **cfg)
    for _ in range(2):
        dt = a.cfl_dt(0.7)
        assert abs(dt - b.cfl_dt(0.7)) <= 1e-6 * dt
        a.step(dt)
        b.step(dt)
        ok, err = close_to(a.get_state(), b.get_state())
        assert ok, err
    a.run(3, 0.7)
    b.run(3, 0.7)
    ok, err = close_to(a.get_state(), b.get_state(), 5e-6)
    assert ok, err
    assert abs(a.time() - b.time()) <= 1e-6 * a.time()
    assert a.tma_sweeps() > 0 and b.tma_sweeps() == 0


@pytest.mark.parametrize("axis", [1, 2])
@pytest.mark.parametrize("kind", [0, 1])
def test_staged_sweep_parity_with_oracle(mhd, axis, kind):
    st = ic.turbulence((64, 32, 24), seed=41, dtype=torch.float64, kmin=1.0, kmax=4.0)
    s = ic.as_oracle_input(st)
    tau = 0.35 / oracle.cfl_rate(s, G)
    nz, ny, nx = st.shape[1:]
    box = mhd.Box(nx, ny, nz, gamma=G)
    box.set_state(to_gpu(st))
    box.sweep(axis, kind, tau)
    assert box.tma_sweeps() == 1
    if kind == 0:
        oracle.fluid_sweep(s, axis, tau, G)
    else:
        oracle.mag_sweep(s, axis, tau)
    err = rel_err(from_gpu(box.get_state()), s, field_scales(s))
    assert np.all(err < 1e-5), err


def test_staged_full_step_parity_with_oracle(mhd):
    """One full step of 64 x 32 x 24 turbulence, every y and z sweep staged:
    within the non-smooth one-step bound (1e-4) of the oracle."""
    st = ic.turbulence((64, 32, 24), seed=43, dtype=torch.float64, kmin=1.0, kmax=4.0)
    s = ic.as_oracle_input(st)
    nz, ny, nx = st.shape[1:]
    box = mhd.Box(nx, ny, nz, gamma=G)
    box.set_state(to_gpu(st))
    dt = oracle.cfl_dt(s, G, 0.7)
    box.step(dt)
    assert box.tma_sweeps() >= 7  # 4 fluid sweeps, 2 magnetic y sweeps, the fused z pair
    oracle.step(s, dt, G)
    err = rel_err(from_gpu(box.get_state()), s, field_scales(s))
    assert np.all(err < 1e-4), err
