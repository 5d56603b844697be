"""The FP64 GPU path (mhd_create_f64) against the FP64 oracle on identical
inputs.  Both compute the Section II.B scheme in double precision, each in
its own operation order, so they agree to a few units of FP64 rounding per
operation, amplified only by the limiter's switches.  Bounds (max error of
each field relative to max(max|oracle_f|, S_f), as in test_gpu_parity):
1e-12 after one step and 1e-10 after 20 steps of the Alfven wave and the
shock tube; single sweeps 1e-13.  The FP64 inputs are not rounded to FP32."""
import numpy as np
import pytest
import torch

import oracle
from paper_1004_1680_gb300 import initial_conditions as ic
from tests.parity_util import G, field_scales, rel_err

pytestmark = pytest.mark.gpu


def _pair(st64):
    from paper_1004_1680_gb300 import mhd
    s = np.ascontiguousarray(st64.cpu().numpy())
    nz, ny, nx = s.shape[1:]
    box = mhd.Box64(nx, ny, nz, gamma=G)
    box.set_state(st64.contiguous().cuda())
    return s, box


@pytest.mark.parametrize("axis", [0, 1, 2])
@pytest.mark.parametrize("kind", [0, 1])
def test_fp64_single_sweeps(axis, kind):
    st = ic.turbulence((20, 12, 28), seed=31, dtype=torch.float64, kmin=1.0, kmax=3.0)
    s, box = _pair(st)
    tau = 0.35 / oracle.cfl_rate(s, G)
    box.sweep(axis, kind, tau)
    if kind == 0:
        oracle.fluid_sweep(s, axis, tau, G)
    else:
        oracle.mag_sweep(s, axis, tau)
    err = rel_err(box.get_state(device="cpu").numpy(), s, field_scales(s))
    assert np.all(err < 1e-13), err


@pytest.mark.parametrize("case", ["alfven", "sod"])
def test_fp64_one_and_twenty_steps(case):
    if case == "alfven":
        st, _ = ic.alfven_wave((32, 32, 32), k_int=(1, 1, 1), amp=1e-6)
    else:
        st = ic.sod((32, 32, 32))
    s, box = _pair(st.to(torch.float64))
    S = field_scales(s)
    for n in range(20):
        dt = oracle.cfl_dt(s, G, 0.7)
        assert abs(box.cfl_dt(0.7) - dt) <= 1e-14 * dt
        oracle.step(s, dt, G)
        box.step(dt)
        if n == 0:
            err1 = rel_err(box.get_state(device="cpu").numpy(), s, S)
            assert np.all(err1 < 1e-12), err1
    err20 = rel_err(box.get_state(device="cpu").numpy(), s, S)
    assert np.all(err20 < 1e-10), err20
    assert box.time() > 0


def test_fp64_device_run_and_unsupported_calls():
    """mhd_run takes its CFL timesteps itself; FP32-only calls are refused."""
    from paper_1004_1680_gb300 import mhd
    st = ic.turbulence((16, 16, 16), seed=2, dtype=torch.float64, kmin=1.0, kmax=2.0)
    s, box = _pair(st)
    box.run(3, 0.7)
    t = 0.0
    for _ in range(3):
        dt = oracle.cfl_dt(s, G, 0.7)
        oracle.step(s, dt, G)
        t += dt
    assert abs(box.time() - t) <= 1e-13 * t
    assert np.all(rel_err(box.get_state(device="cpu").numpy(), s, field_scales(s)) < 1e-12)
    ptrs = mhd._field_ptrs(torch.zeros(8, 1, device="cuda"))
    assert box.lib.mhd_set_state(box.h, ptrs, 1) == mhd.MHD_E_ARG
    assert box.lib.mhd_diagnostics(box.h, (__import__("ctypes").c_double * 10)()) == mhd.MHD_E_ARG
