"""Pins of the oracle's non-periodic boundaries (outflow and reflecting ghost
layers, an extension of the paper's periodic scheme), against results the
mathematics fixes rather than the oracle's own formulas:

* outflow: a single Sod shock tube in the middle of a bounded tube matches
  the exact Riemann solution everywhere, up to the walls (a periodic box, or
  a wrong ghost fill, puts a second Riemann problem at the walls);
* reflecting: a box with reflecting walls evolves exactly like one half of
  the mirror-doubled periodic problem (the scheme is mirror-symmetric, and
  the ghost layers hold exactly the mirror cells), also with magnetic fields;
* reflecting: gas running into a wall stops behind a reflected shock whose
  density is the star density of the symmetric Riemann problem
  (rho, u, p | rho, -u, p).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1004_1680_gb300 import initial_conditions as ic
from tests import exact_riemann as er

G = 5.0 / 3.0
GH = oracle.GHOST


def _advance(s, T, cfl=0.7):
    t = 0.0
    while t < T * (1 - 1e-14):
        dt = min(oracle.cfl_dt(s, G, cfl), T - t)
        oracle.step(s, dt, G)
        t += dt


def _tube(n_int, left, right):
    """A bounded tube along x of n_int interior cells (+ ghosts): primitive
    states left / right of the interior's midpoint, b = 0; returns the state
    and the cell centres (the solver's h = 1 / n over the whole box)."""
    n = n_int + 2 * GH
    x = (np.arange(n) + 0.5) / n
    x0 = (GH + n_int / 2) / n
    s = np.zeros((8, 1, 1, n))
    lefty = x < x0
    rho = np.where(lefty, left[0], right[0])
    u = np.where(lefty, left[1], right[1])
    p = np.where(lefty, left[2], right[2])
    s[0, 0, 0] = rho
    s[1, 0, 0] = rho * u
    s[4, 0, 0] = p / (G - 1.0) + 0.5 * rho * u * u
    return s, x, x0


def test_outflow_single_shock_tube_exact_riemann(oracle_lib):
    WL, WR = (1.0, 0.0, 1.0), (0.125, 0.0, 0.1)
    T = 0.1
    errs = []
    for n_int in (256, 512):
        s, x, x0 = _tube(n_int, WL, WR)
        with oracle.boundaries(x="outflow"):
            _advance(s, T)
        inner = slice(GH, GH + n_int)
        ex = er.sample(WL, WR, G, (x[inner] - x0) / T)
        rho = s[0, 0, 0, inner]
        errs.append(np.mean(np.abs(rho - ex[0])))
        # the states next to the walls are the undisturbed initial ones
        assert abs(rho[0] - WL[0]) < 1e-12 and abs(rho[-1] - WR[0]) < 1e-12
    assert errs[1] < 0.01
    assert errs[1] < 0.7 * errs[0]  # converging


def test_periodic_tube_is_disturbed_at_the_walls(oracle_lib):
    """Control for the test above: the same tube without the outflow fill
    (periodic, ghosts included) develops a second Riemann problem at the
    wrap, so the cells next to the walls leave their initial states."""
    s, x, x0 = _tube(256, (1.0, 0.0, 1.0), (0.125, 0.0, 0.1))
    _advance(s, 0.1)
    assert abs(s[0, 0, 0, GH] - 1.0) > 1e-3


def _mirror_double(half):
    """Periodic state of twice the x extent: `half` (reflecting walls at its
    x faces 0 and nx) followed by its mirror image, m_x and b_x negated."""
    nz, ny, nx = half.shape[1:]
    full = np.zeros((8, nz, ny, 2 * nx))
    full[:, :, :, :nx] = half
    mir = half[:, :, :, ::-1].copy()
    mir[1] *= -1.0
    full[:, :, :, nx:] = mir
    # faces: b_x at face nx + m mirrors face nx - m, negated (face nx = wall)
    bx = half[5]
    full[5, :, :, nx] = 0.0
    for m in range(1, nx):
        full[5, :, :, nx + m] = -bx[:, :, nx - m]
    return full


@pytest.mark.parametrize("magnetic", [False, True])
def test_reflecting_walls_equal_the_mirror_doubled_periodic_box(oracle_lib, magnetic):
    # the solver's cell width is 1 / n of the whole box, so the doubled box
    # (2 nx cells) and the box with ghost layers (nx + 2 GH) need the same n
    nx, ny, nz = 2 * GH, 12, 10
    st = ic.turbulence((nx, ny, nz), seed=11, dtype=torch.float64, kmin=1.0, kmax=3.0)
    half = st.numpy().copy()
    if not magnetic:
        half[5:8] = 0.0
    half[5, :, :, 0] = 0.0  # the walls carry no normal field
    full = _mirror_double(half)
    # the same half inside a box with reflecting x walls and ghost layers
    box = np.zeros((8, nz, ny, nx + 2 * GH))
    box[:, :, :, GH:GH + nx] = half
    box[5, :, :, GH + nx] = 0.0  # high wall face
    dts = []
    for _ in range(4):
        dts.append(oracle.cfl_dt(full, G, 0.6))
        oracle.step(full, dts[-1], G)
    with oracle.boundaries(x="reflecting"):
        for n in range(4):
            # the rate over the interior equals the doubled box's (mirror cells)
            assert oracle.cfl_dt(box, G, 0.6) == pytest.approx(dts[n], rel=1e-13)
            oracle.step(box, dts[n], G)
    got = box[:, :, :, GH:GH + nx]
    want = full[:, :, :, :nx]
    scale = np.max(np.abs(want), axis=(1, 2, 3)) + 1e-30
    err = np.max(np.abs(got - want), axis=(1, 2, 3)) / scale
    assert np.all(err < 1e-12), err
    # the wall faces keep no normal field
    assert np.max(np.abs(box[5, :, :, GH])) < 1e-13
    assert np.max(np.abs(box[5, :, :, GH + nx])) < 1e-13


def test_reflecting_wall_stops_the_gas_behind_the_exact_reflected_shock(oracle_lib):
    """Both halves of a tube run into their walls (u = -u0 left, +u0 right;
    subsonic, so the rarefaction in the middle keeps p > 0).  At each wall the
    gas stops behind a shock with the star state of the symmetric Riemann
    problem (rho0, u0, p0 | rho0, -u0, p0)."""
    rho0, u0, p0 = 1.0, 0.3, 1.0
    n_int = 400
    n = n_int + 2 * GH
    x = (np.arange(n) + 0.5) / n
    mid = (GH + n_int / 2) / n
    u = np.where(x < mid, -u0, u0)
    s = np.zeros((8, 1, 1, n))
    s[0] = rho0
    s[1, 0, 0] = rho0 * u
    s[4] = p0 / (G - 1.0) + 0.5 * rho0 * u0 * u0
    T = 0.1
    with oracle.boundaries(x="reflecting"):
        _advance(s, T)
    ps, us = er.star_state((rho0, u0, p0), (rho0, -u0, p0), G)
    assert abs(us) < 1e-12
    mu = (G - 1.0) / (G + 1.0)
    rs = rho0 * (ps / p0 + mu) / (mu * ps / p0 + 1.0)  # Rankine-Hugoniot density
    S = rho0 * u0 / (rho0 - rs)  # mass across the shock: rho0 (u0 - S) = rs (0 - S)
    wall = (GH + n_int) / n
    xs = wall + S * T  # S < 0: the right wall's shock runs back into the gas
    xi = x[GH:GH + n_int]
    rho = s[0, 0, 0, GH:GH + n_int]
    vel = s[1, 0, 0, GH:GH + n_int] / rho
    behind = (xi > xs + 0.02) & (xi < wall - 0.01)
    head = mid + (u0 + np.sqrt(G * p0 / rho0)) * T  # head of the middle rarefaction
    ahead = (xi < xs - 0.02) & (xi > head + 0.02)
    assert behind.sum() > 10 and ahead.sum() > 10
    assert np.allclose(rho[behind], rs, rtol=0.01)
    assert np.max(np.abs(vel[behind])) < 0.01 * u0 * 10
    assert np.allclose(rho[ahead], rho0, rtol=1e-3)
    # the jump sits where the exact shock is (within a few cells)
    right = xi > head + 0.02
    i = np.argmax(np.abs(np.diff(rho[right])))
    xr = xi[right]
    assert abs(0.5 * (xr[i] + xr[i + 1]) - xs) < 4.0 / n
    # mirror symmetry of the whole tube
    assert np.allclose(rho, rho[::-1], rtol=1e-12, atol=1e-12)


def test_fill_rules_on_a_small_array(oracle_lib):
    """The fill copies only interior and wall values, on both ends."""
    rng = np.random.default_rng(0)
    s = rng.standard_normal((8, 2, 3, 14))
    with oracle.boundaries(x="outflow"):
        oracle.fill_ghosts(s)
    assert np.all(s[0, :, :, :GH] == s[0, :, :, GH:GH + 1])
    assert np.all(s[0, :, :, -GH:] == s[0, :, :, -GH - 1:-GH])
    assert np.all(s[5, :, :, :GH] == s[5, :, :, GH:GH + 1])            # normal faces copy the wall
    assert np.all(s[5, :, :, 14 - GH + 1:] == s[5, :, :, 14 - GH:14 - GH + 1])
    s = rng.standard_normal((8, 2, 14, 5))
    with oracle.boundaries(y="reflecting"):
        oracle.fill_ghosts(s)
    for k in range(GH):
        assert np.all(s[0, :, k, :] == s[0, :, 2 * GH - 1 - k, :])
        assert np.all(s[2, :, k, :] == -s[2, :, 2 * GH - 1 - k, :])    # normal momentum
        assert np.all(s[1, :, k, :] == s[1, :, 2 * GH - 1 - k, :])     # tangential momentum
        assert np.all(s[6, :, k, :] == -s[6, :, 2 * GH - k, :])        # normal faces mirror the wall
        assert np.all(s[5, :, k, :] == s[5, :, 2 * GH - 1 - k, :])     # tangential faces as cells


def test_short_non_periodic_axis_is_refused(oracle_lib):
    s = np.ones((8, 2, 3, 14))
    with oracle.boundaries(y="outflow"):
        with pytest.raises(ValueError):
            oracle.fill_ghosts(s)
        with pytest.raises(ValueError):
            oracle.step(s, 0.01, G)
