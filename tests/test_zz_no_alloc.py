"""mhd_diagnostics_static: the FP64 diagnostics for callers that cannot
allocate device memory (for example code running where another allocator
owns the device memory, or where a cudaMalloc would synchronise a
latency-critical loop).  It uses a fixed scratch array inside the library
instead of memory from mhd_create; its results must match mhd_diagnostics on
the same state, on consecutive calls (the shared array keeps the previous
call's contents).  This file is collected last on purpose."""
import math

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def test_static_diagnostics_match_the_allocating_entry_point():
    """Both entry points run the same kernels with the same grid on the same
    state, so their results agree bit for bit.  112^3 has more cells than the
    diagnostics grid covers without looping (1216 blocks of 1024 cells): it
    uses the capped grid, whose partials end exactly where the results begin
    in the fixed array."""
    from paper_1004_1680_gb300 import initial_conditions as ic
    from paper_1004_1680_gb300 import mhd
    for dims, seed in (((48, 40, 36), 1), ((32, 24, 20), 2), ((112, 112, 112), 3)):
        st = ic.turbulence(dims, seed=seed, dtype=torch.float32, kmin=1.0, kmax=3.0).contiguous().cuda()
        box = mhd.Box(*dims)
        box.set_state(st)
        box.run(2, 0.7)
        cur = box.get_state()                      # the state both entry points see
        ref = box.diagnostics()
        s = cur.double().cpu().numpy()
        for _ in range(2):                          # two calls in a row
            got = mhd.diagnostics_static(cur, gamma=box.gamma)
            assert np.array_equal(got, ref), (dims, got - ref)
            # and both are the exactly rounded sums within the stated bound
            for q in range(8):
                exact = math.fsum(s[q].ravel().tolist())
                assert abs(got[q] - exact) <= 1e-13 * float(np.sum(np.abs(s[q]))) + 1e-300
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
