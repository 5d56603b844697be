"""mhd_diagnostics_static: the FP64 diagnostics for callers that cannot
allocate device memory (for example code running where another allocator
owns the device memory, or where a cudaMalloc would synchronise a
latency-critical loop).  It uses a fixed scratch array inside the library
instead of memory from mhd_create; its results must match mhd_diagnostics on
the same state, on consecutive calls (the shared array keeps the previous
call's contents).  This file is collected last on purpose."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def test_static_diagnostics_match_the_allocating_entry_point():
    from paper_1004_1680_gb300 import initial_conditions as ic
    from paper_1004_1680_gb300 import mhd
    for dims, seed in (((48, 40, 36), 1), ((32, 24, 20), 2)):
        st = ic.turbulence(dims, seed=seed, dtype=torch.float32, kmin=1.0, kmax=3.0).contiguous().cuda()
        box = mhd.Box(*dims)
        box.set_state(st)
        box.run(2, 0.7)
        cur = box.get_state()                      # the state both entry points see
        ref = box.diagnostics()
        for _ in range(2):                          # two calls in a row
            got = mhd.diagnostics_static(cur, gamma=box.gamma)
            s = cur.double().cpu().numpy()
            for q in range(8):
                assert abs(got[q] - ref[q]) <= 1e-13 * float(np.sum(np.abs(s[q]))) + 1e-300
            assert got[8] == pytest.approx(ref[8], rel=1e-9, abs=1e-14)
            assert got[9] == pytest.approx(ref[9], rel=1e-12)
        box.close()


def test_static_diagnostics_rejects_oversized_boxes():
    from paper_1004_1680_gb300 import mhd
    lib = mhd.load()
    import ctypes
    ptrs = (ctypes.c_void_p * 8)(*[1] * 8)
    out = (ctypes.c_double * 10)()
    rc = lib.mhd_diagnostics_static(2048, 1024, 1024, 5.0 / 3.0, ptrs, out, None)
    assert rc == mhd.MHD_E_ARG
    assert b"too large" in lib.mhd_last_error()
