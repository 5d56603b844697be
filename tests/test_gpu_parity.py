"""GPU (FP32, through the C ABI) against the FP64 oracle on identical seeded inputs.

Tolerances (max relative field error, each field normalised by
max(max|oracle_f|, S_f) with the background scales S_f of parity_util):
  * one sweep or one full step of a smooth problem: <= 1e-5;
  * 20 full steps of a smooth problem: <= 1e-3;
  * non-smooth problems (shock tube, turbulence): <= 1e-4 after one step and
    mean-absolute <= 1e-4 after 20 steps.
FP32 rounding of one full step leaves about 1e-7 relative per cell; the
bounds allow the growth of that rounding through 12 sweeps of a limited
scheme (whose limiter switches are continuous), not any systematic error.
"""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_1004_1680_gb300 import initial_conditions as ic
from tests.parity_util import G, field_scales, from_gpu, l1_rel, rel_err, sub_block, to_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mhd():
    from paper_1004_1680_gb300 import mhd as m
    m.load()
    return m


def make_box(mhd, st64):
    nz, ny, nx = st64.shape[1:]
    box = mhd.Box(nx, ny, nz, gamma=G)
    box.set_state(to_gpu(st64))
    return box


def oracle_input(st64):
    return ic.as_oracle_input(st64)


# --------------------------------------------------------------------------
# single sweeps, every axis and kind, on a non-cubic box with ragged tiles

@pytest.mark.parametrize("axis", [0, 1, 2])
@pytest.mark.parametrize("kind", [0, 1])
def test_single_sweep_parity(mhd, axis, kind):
    st = ic.turbulence((48, 40, 36), seed=21, dtype=torch.float64, kmin=1.0, kmax=4.0)
    s = oracle_input(st)
    tau = 0.35 / oracle.cfl_rate(s, G)
    box = make_box(mhd, st)
    box.sweep(axis, kind, tau)
    g = from_gpu(box.get_state())
    if kind == 0:
        oracle.fluid_sweep(s, axis, tau, G)
    else:
        oracle.mag_sweep(s, axis, tau)
    err = rel_err(g, s, field_scales(s))
    assert np.all(err < 1e-5), err


@pytest.mark.parametrize("xpath", [1, 2])
@pytest.mark.parametrize("kind", [0, 1])
def test_x_sweep_both_paths(mhd, xpath, kind):
    """x sweeps read directly (path 1) or through the x<->y exchanged copy
    (path 2); both against the oracle, on boxes with ragged tiles and a short
    (< 16 cell) x axis."""
    for dims in ((48, 40, 36), (12, 20, 8)):
        st = ic.turbulence(dims, seed=23, dtype=torch.float64, kmin=1.0, kmax=3.0)
        s = oracle_input(st)
        tau = 0.35 / oracle.cfl_rate(s, G)
        box = make_box(mhd, st)
        box.set_xpath(xpath)
        box.sweep(0, kind, tau)
        g = from_gpu(box.get_state())
        if kind == 0:
            oracle.fluid_sweep(s, 0, tau, G)
        else:
            oracle.mag_sweep(s, 0, tau)
        err = rel_err(g, s, field_scales(s))
        assert np.all(err < 1e-5), (dims, err)


@pytest.mark.parametrize("xpath", [1, 2, 3])
def test_full_steps_both_x_paths(mhd, xpath):
    st = ic.turbulence((40, 24, 20), seed=24, dtype=torch.float64, kmin=1.0, kmax=3.0)
    s = oracle_input(st)
    S = field_scales(s)
    box = make_box(mhd, st)
    box.set_xpath(xpath)
    t_orc, _ = oracle.run(s, 4, 0.7, G)
    box.run(4, 0.7)
    assert box.time() == pytest.approx(t_orc, rel=1e-5)
    err = rel_err(from_gpu(box.get_state()), s, S)
    assert np.all(err < 1e-4), err


@pytest.mark.parametrize("axis", [0, 1, 2])
@pytest.mark.parametrize("kind", [0, 1])
def test_paper_data_flow_single_sweeps(mhd, axis, kind):
    """x path 3 (every sweep along the contiguous axis of a transposed copy)
    against the oracle, one sweep of each axis and kind on a box whose three
    extents differ."""
    st = ic.turbulence((48, 40, 36), seed=25, dtype=torch.float64, kmin=1.0, kmax=3.0)
    s = oracle_input(st)
    tau = 0.35 / oracle.cfl_rate(s, G)
    box = make_box(mhd, st)
    box.set_xpath(3)
    box.sweep(axis, kind, tau)
    g = from_gpu(box.get_state())
    if kind == 0:
        oracle.fluid_sweep(s, axis, tau, G)
    else:
        oracle.mag_sweep(s, axis, tau)
    assert np.all(rel_err(g, s, field_scales(s)) < 1e-5)


@pytest.mark.parametrize("segs", [(16, 8, 12), (8, 20, 4), (48, 40, 36)])
def test_segmentation_is_bitwise_neutral(mhd, segs):
    st = ic.turbulence((48, 40, 36), seed=22, dtype=torch.float64, kmin=1.0, kmax=4.0)
    a = make_box(mhd, st)
    b = make_box(mhd, st)
    b.set_segments(*segs)
    dt = a.cfl_dt(0.7)
    a.step(dt)
    b.step(dt)
    assert torch.equal(a.get_state(), b.get_state())


@pytest.mark.parametrize("dims,segs", [((48, 40, 36), None), ((40, 36, 36), (8, 12, 12)),
                                       ((32, 24, 8), None), ((12, 5, 3), None), ((64, 16, 96), (16, 16, 16))])
def test_fused_z_magnetic_pair_is_bitwise_two_sweeps(mhd, dims, segs):
    """The two middle z magnetic sweeps of a step in one launch give bitwise
    the state of two launches: ragged tiles, z shorter than 16 (periodic
    images of the warm-up wrap more than once), segmented pencils."""
    st = ic.turbulence(dims, seed=23, dtype=torch.float64, kmin=1.0, kmax=1.0 if min(dims) < 8 else 3.0,
                       mach=0.5)
    a = make_box(mhd, st)
    b = make_box(mhd, st)
    b.set_fusion(False)
    if segs:
        a.set_segments(*segs)
        b.set_segments(*segs)
    for _ in range(3):
        dt = a.cfl_dt(0.7)
        assert dt == b.cfl_dt(0.7)
        a.step(dt)
        b.step(dt)
        assert torch.equal(a.get_state(), b.get_state())
    a.run(2, 0.7)
    b.run(2, 0.7)
    assert torch.equal(a.get_state(), b.get_state())
    assert a.time() == b.time()


# --------------------------------------------------------------------------
# full steps on the small workloads: 32^3 Alfven wave and 32^3 shock tube

def test_alfven_32_one_and_twenty_steps(mhd):
    st, info = ic.alfven_wave((32, 32, 32), k_int=(1, 1, 1), amp=1e-6)
    s = oracle_input(st)
    S = field_scales(s)
    box = make_box(mhd, st)
    for n in range(20):
        dt = oracle.cfl_dt(s, G, 0.7)
        oracle.step(s, dt, G)
        box.step(dt)
        if n == 0:
            err1 = rel_err(from_gpu(box.get_state()), s, S)
            assert np.all(err1 < 1e-5), err1
    err20 = rel_err(from_gpu(box.get_state()), s, S)
    assert np.all(err20 < 1e-3), err20


def test_alfven_perturbation_amplitude_1e4(mhd):
    """The wave itself (not only the background) agrees: amplitude 1e-4 so
    that FP32 resolves it; error of the velocity perturbation relative to
    its amplitude after 20 steps."""
    amp = 1e-4
    st, info = ic.alfven_wave((32, 32, 32), k_int=(1, 1, 1), amp=amp)
    s = oracle_input(st)
    box = make_box(mhd, st)
    for _ in range(20):
        dt = oracle.cfl_dt(s, G, 0.7)
        oracle.step(s, dt, G)
        box.step(dt)
    g = from_gpu(box.get_state())
    assert np.max(np.abs(g[1:4] - s[1:4])) / amp < 2e-2


def test_sod_32_cubed(mhd):
    st = ic.sod((32, 32, 32), axis=0)
    s = oracle_input(st)
    S = field_scales(s)
    box = make_box(mhd, st)
    for n in range(20):
        dt = oracle.cfl_dt(s, G, 0.7)
        oracle.step(s, dt, G)
        box.step(dt)
        if n == 0:
            err1 = rel_err(from_gpu(box.get_state()), s, S)
            assert np.all(err1 < 1e-4), err1
    l1 = l1_rel(from_gpu(box.get_state()), s, S)
    assert np.all(l1 < 1e-4), l1


def test_turbulence_odd_box_steps(mhd):
    st = ic.turbulence((20, 12, 28), seed=5, dtype=torch.float64, kmin=1.0, kmax=3.0)
    s = oracle_input(st)
    S = field_scales(s)
    box = make_box(mhd, st)
    for n in range(10):
        dt = oracle.cfl_dt(s, G, 0.7)
        oracle.step(s, dt, G)
        box.step(dt)
        if n == 0:
            err1 = rel_err(from_gpu(box.get_state()), s, S)
            assert np.all(err1 < 1e-5), err1
    l1 = l1_rel(from_gpu(box.get_state()), s, S)
    assert np.all(l1 < 1e-4), l1


@pytest.mark.parametrize("dims", [(4, 1, 1), (8, 1, 1), (4, 3, 5), (64, 1, 2), (12, 32, 1)])
def test_degenerate_boxes(mhd, dims):
    """Minimum sizes, 1- and 2-D boxes (pencils of length 1)."""
    st = ic.turbulence(dims, seed=3, dtype=torch.float64, kmin=1.0, kmax=1.0, mach=0.5)
    s = oracle_input(st)
    S = field_scales(s)
    box = make_box(mhd, st)
    for _ in range(3):
        dt = oracle.cfl_dt(s, G, 0.7)
        oracle.step(s, dt, G)
        box.step(dt)
    err = rel_err(from_gpu(box.get_state()), s, S)
    assert np.all(err < 1e-5), err


# --------------------------------------------------------------------------
# CFL, device-resident timestep, time, diagnostics

def test_cfl_dt_and_device_resident_run(mhd):
    st = ic.turbulence((32, 24, 16), seed=8, dtype=torch.float64, kmin=1.0, kmax=3.0)
    s = oracle_input(st)
    box = make_box(mhd, st)
    assert box.cfl_dt(0.7) == pytest.approx(oracle.cfl_dt(s, G, 0.7), rel=2e-6)
    t_orc, dts = oracle.run(s, 5, 0.7, G)
    box.run(5, 0.7)
    assert box.time() == pytest.approx(t_orc, rel=1e-5)
    err = rel_err(from_gpu(box.get_state()), s, field_scales(s))
    assert np.all(err < 1e-4), err
    # the rate left by the fused epilogue equals a fresh reduction of the same state
    assert box.cfl_dt(0.7) == pytest.approx(oracle.cfl_dt(s, G, 0.7), rel=1e-5)


def test_diagnostics_fp64(mhd):
    st = ic.orszag_tang((32, 32, 32))
    box = make_box(mhd, st)
    box.run(3, 0.7)
    g = box.get_state()
    s = from_gpu(g)                      # the exact FP32 state, widened
    d_gpu = box.diagnostics()
    d_orc = oracle.diagnostics(s, G)
    for q in range(8):
        scale = np.sum(np.abs(s[q]))
        assert abs(d_gpu[q] - d_orc[q]) <= 1e-13 * scale + 1e-300
    assert d_gpu[8] == pytest.approx(d_orc[8], rel=1e-9, abs=1e-14)
    assert d_gpu[9] == pytest.approx(d_orc[9], rel=1e-12)
    assert np.array_equal(box.diagnostics(), d_gpu)      # fixed-order reduction


def _hard_diag_state(shape, seed):
    """An FP32 state built to stress the diagnostics (as FP64 holding FP32
    values): momentum spanning 20 decades with both signs, face fields with
    subnormal values and signed zeros, and pressures within ~1e-7 of 1
    everywhere (FP32 estimates cannot separate them, so the exact FP64
    extremum has to be found among many candidates), plus one isolated low
    pressure and one isolated div b spike."""
    nx, ny, nz = shape
    rng = np.random.default_rng(seed)
    s = np.empty((8, nz, ny, nx))
    s[0] = 1.0 + 0.5 * rng.random((nz, ny, nx))
    s[1:4] = rng.standard_normal((3, nz, ny, nx)) * 10.0 ** rng.integers(-20, 1, (3, nz, ny, nx))
    s[5:8] = 0.1 * rng.standard_normal((3, nz, ny, nx))
    s[5, 0, 0, :7] = np.array([1e-40, -1e-41, 0.0, -0.0, 1e-45, -1e-45, 3e-39])
    s[7, 1, 2, 3] += 0.5          # div b spike in two cells (its faces)
    s = s.astype(np.float32).astype(np.float64)
    # total energy for p = 1 (+ 1e-9 noise, lost to FP32 rounding)
    kin = 0.5 * np.sum(s[1:4] ** 2, axis=0) / s[0]
    bc = [0.5 * (s[5 + d] + np.roll(s[5 + d], -1, axis=2 - d)) for d in range(3)]
    mag = 0.5 * sum(b * b for b in bc)
    p = 1.0 + 1e-9 * rng.random((nz, ny, nx))
    p[nz // 2, 3, 5] = 0.25
    s[4] = p / (G - 1.0) + kin + mag
    return s.astype(np.float32).astype(np.float64)


@pytest.mark.parametrize("shape", [(40, 24, 36), (36, 7, 5)])
def test_diagnostics_on_hard_inputs(mhd, shape):
    """Sums within 1e-13 of sum|f| of the exactly rounded sums; max |div b| and
    min p equal to the FP64 evaluation of every cell (the kernel evaluates
    FP64 only where an FP32 bound cannot rule a cell out)."""
    s = _hard_diag_state(shape, seed=11)
    nx, ny, nz = shape
    box = mhd.Box(nx, ny, nz, gamma=G)
    box.set_state(torch.from_numpy(s).to(torch.float32).cuda())
    d = box.diagnostics()
    o = oracle.diagnostics(s, G)
    for q in range(8):
        assert abs(d[q] - o[q]) <= 1e-13 * np.sum(np.abs(s[q])) + 1e-300, q
    assert d[8] == pytest.approx(o[8], rel=1e-13)
    assert d[9] == pytest.approx(o[9], rel=1e-13)
    assert d[9] == pytest.approx(0.25, rel=1e-5)
    # the near-tied pressures: remove the isolated minimum, the exact minimum
    # of the rest must still be found
    s2 = s.copy()
    s2[4, nz // 2, 3, 5] = s2[4, nz // 2, 3, 4]
    box.set_state(torch.from_numpy(s2).to(torch.float32).cuda())
    d2 = box.diagnostics()
    o2 = oracle.diagnostics(s2, G)
    assert d2[9] == pytest.approx(o2[9], rel=1e-12)
    # a NaN propagates into its field's sum, as in an FP64 sum
    s2[0, 0, 0, 0] = np.nan
    box.set_state(torch.from_numpy(s2).to(torch.float32).cuda())
    assert np.isnan(box.diagnostics()[0])
    box.close()


def test_conservation_and_div_b_on_gpu(mhd):
    st = ic.turbulence((64, 64, 64), seed=2, dtype=torch.float64, kmin=1.0, kmax=4.0)
    box = make_box(mhd, st)
    d0 = box.diagnostics()
    bmax = float(torch.max(torch.abs(st[5:8])))
    box.run(10, 0.7)
    d1 = box.diagnostics()
    s = from_gpu(box.get_state())
    for q in (0, 4):
        assert abs(d1[q] - d0[q]) / abs(d0[q]) < 1e-6
    absm = np.sum(np.abs(s[1:4]))
    for q in (1, 2, 3):
        assert abs(d1[q] - d0[q]) / absm < 1e-6
    # FP32 face values carry ~1e-7 relative rounding; CT keeps div b at that level
    assert d1[8] < 1e-5 * bmax
    assert d1[9] > 0


# --------------------------------------------------------------------------
# symmetry, determinism, restart

def test_cyclic_permutation_per_sweep(mhd):
    from tests.test_oracle_pins import cycle, uncycle
    st = ic.turbulence((16, 12, 20), seed=4, dtype=torch.float64, kmin=1.0, kmax=3.0)
    s = oracle_input(st)
    tau = 0.4 / oracle.cfl_rate(s, G)
    for d_orig, k in ((1, 1), (2, 2)):
        a = make_box(mhd, st)
        a.sweep(d_orig, 0, tau)
        a.sweep(d_orig, 1, tau)
        ga = from_gpu(a.get_state())
        c = s.copy()
        for _ in range(k):
            c = cycle(c)
        b = make_box(mhd, torch.from_numpy(c))
        b.sweep(0, 0, tau)
        b.sweep(0, 1, tau)
        gb = from_gpu(b.get_state())
        for _ in range(k):
            gb = uncycle(gb)
        S = field_scales(s)
        assert np.all(rel_err(ga, gb, S) < 1e-6)


def test_bitwise_determinism_and_restart(mhd):
    st = ic.turbulence((32, 32, 32), seed=6, dtype=torch.float64, kmin=1.0, kmax=4.0)
    a = make_box(mhd, st)
    a.run(6, 0.7)
    fa = a.get_state().clone()
    b = make_box(mhd, st)
    b.run(6, 0.7)
    assert torch.equal(fa, b.get_state())
    c = make_box(mhd, st)
    c.run(2, 0.7)
    ck = c.get_state().clone()
    c2 = make_box(mhd, st)
    c2.set_state(ck)
    c2.run(4, 0.7)
    assert torch.equal(fa, c2.get_state())


# --------------------------------------------------------------------------
# full-size workloads, checked on samples the oracle can compute

def test_orszag_tang_256_first_step_full_parity(mhd):
    """256^3 Orszag-Tang vortex: step 1 on the GPU against the whole oracle step."""
    st = ic.orszag_tang((256, 256, 256))
    s = oracle_input(st)
    box = make_box(mhd, st)
    dt = box.cfl_dt(0.7)
    assert dt == pytest.approx(oracle.cfl_dt(s, G, 0.7), rel=2e-6)
    box.step(dt)
    oracle.step(s, dt, G)
    err = rel_err(from_gpu(box.get_state()), s, field_scales(s))
    assert np.all(err < 1e-5), err


def _sub_block_dev(t, lo, size):
    """Periodic sub-block of a device state (as sub_block), copied to the host."""
    idx = [torch.arange(lo[d], lo[d] + size[d], device=t.device) % t.shape[3 - d] for d in range(3)]
    return t.index_select(1, idx[2]).index_select(2, idx[1]).index_select(3, idx[0]).cpu().numpy()


@pytest.mark.parametrize("n", [512, 1024])
def test_turbulence_full_size_sampled_sub_blocks(mhd, n):
    """512^3 and 1024^3 decaying turbulence (the bench workloads), one step in
    the bench's launch configuration; the oracle steps periodic sub-blocks
    with a 24-cell halo (one full step reaches 14 cells) and the interiors
    are compared.  Sub-blocks are cut on the device, so the 34 GB state of
    the 1024^3 box never goes to the host."""
    box = mhd.Box(n, n, n, gamma=G)  # before the input, as bench.py does (its buffers first)
    st32 = ic.turbulence((n, n, n), seed=0, device="cuda", dtype=torch.float32)
    box.set_state(st32)
    torch.cuda.empty_cache()
    dt = box.cfl_dt(0.7)
    box.step(dt)
    out = box.get_state()
    H, L = 24, 24
    rng = np.random.default_rng(0)
    corners = [(0, 0, 0), (n - L, n - L, n - L)] + [tuple(int(c) for c in rng.integers(0, n, 3)) for _ in range(3)]
    try:
        for lo in corners:
            nb = L + 2 * H
            blk = _sub_block_dev(st32, [c - H for c in lo], [nb] * 3).astype(np.float64)
            S = field_scales(blk)
            # the sub-box is a unit cube of nb cells: scale dt so tau/h is unchanged
            oracle.step(blk, dt * n / nb, G)
            ref = blk[:, H:H + L, H:H + L, H:H + L]
            got = _sub_block_dev(out, lo, [L] * 3)
            err = rel_err(got.astype(np.float64), ref, S)
            assert np.all(err < 1e-5), (lo, err)
    finally:
        del st32, out
        box.close()
        torch.cuda.empty_cache()


def test_pressure_floor_parity(mhd):
    """Optional pressure floor on a strongly magnetised box that loses
    positivity without it: GPU and oracle with the same floor agree."""
    sp = ic.ensemble_specs(256, seed=2024)[8]
    st = ic.turbulence(sp["dims"], seed=sp["seed"], mach=sp["mach"], beta=sp["beta"],
                       dtype=torch.float64)
    s = oracle_input(st)
    S = field_scales(s)
    box = make_box(mhd, st)
    box.set_pressure_floor(1e-3)
    oracle.set_pressure_floor(1e-3)
    try:
        for n in range(6):
            dt = oracle.cfl_dt(s, G, 0.7)
            oracle.step(s, dt, G)
            box.step(dt)
        g = from_gpu(box.get_state())
    finally:
        oracle.set_pressure_floor(0.0)
    assert np.min(oracle.pressure(g, G)) > 0.9e-3
    err = rel_err(g, s, S)
    l1 = l1_rel(g, s, S)
    assert np.all(err < 1e-3), err
    assert np.all(l1 < 1e-4), l1


def test_invalid_state_is_reported(mhd):
    st = ic.uniform((8, 8, 8), rho=1.0, p=1.0)
    st[0, 2, 3, 4] = -1.0
    box = make_box(mhd, st)
    with pytest.raises(mhd.MHDError) as e:
        box.cfl_dt(0.7)
    assert e.value.code == mhd.MHD_E_STATE
