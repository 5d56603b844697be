"""Sweeps along x over whole staged rows (x path 1 on boxes whose x extent is
a multiple of 128, up to 2048) against the pencil sweeps and the FP64 oracle.

The row sweeps do the arithmetic of the pencil sweeps cell by cell: the fluid
row sweep takes the freezing speeds' square roots from the hardware
approximation, as the TMA-staged strided sweeps do (agreement with the
register-load sweep to FP32 rounding); the magnetic row sweep has no square
root and must match the register-load sweep bitwise.  `set_tma(False)`
selects the pencil sweeps for comparison.
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


def pair(mhd, st64, scheme=None, floor=None):
    nz, ny, nx = st64.shape[1:]
    boxes = []
    for rows in (True, False):
        b = mhd.Box(nx, ny, nz, gamma=G)
        b.set_xpath(1)
        b.set_tma(rows)
        if scheme:
            b.set_scheme(*scheme)
        if floor:
            b.set_pressure_floor(floor)
        b.set_state(to_gpu(st64))
        boxes.append(b)
    return boxes


def close_to(a, b, tol=1e-6):
    """max per-field |a - b| / field scale, the scales of the FP64 state a"""
    sa = a.to(torch.float64).cpu().numpy()
    err = rel_err(b.to(torch.float64).cpu().numpy(), sa, field_scales(sa))
    return bool(np.all(err < tol)), err


DIMS = [(128, 16, 8), (256, 12, 10), (128, 9, 7), (384, 8, 8), (1024, 6, 4)]


@pytest.mark.parametrize("dims", DIMS)
def test_fluid_row_sweep_matches_the_pencil_sweep(mhd, dims):
    st = ic.turbulence(dims, seed=51, dtype=torch.float64, kmin=1.0, kmax=4.0)
    a, b = pair(mhd, st)
    tau = 0.35 / oracle.cfl_rate(ic.as_oracle_input(st), G)
    a.sweep(0, 0, tau)
    b.sweep(0, 0, tau)
    assert a.tma_sweeps() == 1
    ok, err = close_to(a.get_state(), b.get_state())
    assert ok, err


# the magnetic row sweep needs nx up to 1024 and ny a multiple of its tile's
# rows (4; 2 for rows longer than 512)
MAG_DIMS = [(128, 16, 8), (256, 12, 10), (384, 8, 8), (128, 4, 3), (512, 8, 16), (1024, 6, 4), (896, 2, 5)]


@pytest.mark.parametrize("dims", MAG_DIMS)
def test_mag_row_sweep_matches_the_pencil_sweep_bitwise(mhd, dims):
    st = ic.turbulence(dims, seed=61, dtype=torch.float64, kmin=1.0, kmax=4.0)
    a, b = pair(mhd, st)
    tau = 0.35 / oracle.cfl_rate(ic.as_oracle_input(st), G)
    a.sweep(0, 1, tau)
    b.sweep(0, 1, tau)
    assert a.tma_sweeps() == 1 and b.tma_sweeps() == 0
    assert torch.equal(a.get_state(), b.get_state())


@pytest.mark.parametrize("dims", MAG_DIMS[:2])
def test_mag_row_sweep_parity_with_oracle(mhd, dims):
    st = ic.turbulence(dims, seed=63, dtype=torch.float64, kmin=1.0, kmax=4.0)
    s = ic.as_oracle_input(st)
    tau = 0.35 / oracle.cfl_rate(s, G)
    nz, ny, nx = st.shape[1:]
    box = mhd.Box(nx, ny, nz, gamma=G)
    box.set_xpath(1)
    box.set_state(to_gpu(st))
    box.sweep(0, 1, tau)
    assert box.tma_sweeps() == 1
    oracle.mag_sweep(s, 0, tau)
    err = rel_err(from_gpu(box.get_state()), s, field_scales(s))
    assert np.all(err < 1e-5), err


@pytest.mark.parametrize("dims", DIMS[:2])
def test_fluid_row_sweep_parity_with_oracle(mhd, dims):
    st = ic.turbulence(dims, seed=53, dtype=torch.float64, kmin=1.0, kmax=4.0)
    s = ic.as_oracle_input(st)
    tau = 0.35 / oracle.cfl_rate(s, G)
    nz, ny, nx = st.shape[1:]
    box = mhd.Box(nx, ny, nz, gamma=G)
    box.set_xpath(1)
    box.set_state(to_gpu(st))
    box.sweep(0, 0, tau)
    assert box.tma_sweeps() == 1
    oracle.fluid_sweep(s, 0, tau, G)
    err = rel_err(from_gpu(box.get_state()), s, field_scales(s))
    assert np.all(err < 1e-5), err


@pytest.mark.parametrize("scheme, floor", [
    (None, None),
    (("minmod", "bound"), 1e-3),
    (("minmod", "bound"), None),
    (("superbee", "bound"), None),
    (("vanleer", "fast"), None),
    (None, 1e-3),
])
def test_row_steps_match_the_pencil_steps(mhd, scheme, floor):
    """Full steps (the last x sweep carries the fused CFL rate)."""
    st = ic.turbulence((128, 12, 10), seed=57, dtype=torch.float64, kmin=1.0, kmax=3.0, mach=0.8)
    a, b = pair(mhd, st, scheme, floor)
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
    assert a.tma_sweeps() > 0


def test_row_step_parity_with_oracle(mhd):
    """One full step of 128 x 12 x 10 turbulence on x path 1: within the
    non-smooth one-step bound (1e-4) of the oracle."""
    st = ic.turbulence((128, 12, 10), seed=59, dtype=torch.float64, kmin=1.0, kmax=4.0)
    s = ic.as_oracle_input(st)
    nz, ny, nx = st.shape[1:]
    box = mhd.Box(nx, ny, nz, gamma=G)
    box.set_xpath(1)
    box.set_state(to_gpu(st))
    dt = oracle.cfl_dt(s, G, 0.7)
    box.step(dt)
    oracle.step(s, dt, G)
    err = rel_err(from_gpu(box.get_state()), s, field_scales(s))
    assert np.all(err < 1e-4), err
