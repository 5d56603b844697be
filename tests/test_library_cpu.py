"""CPU-side checks of the CUDA library: it builds for sm_103a, loads, exports
every function declared in include/mhd.h, and rejects bad arguments before
touching the GPU.  No compute call is made here."""
import ctypes
import os
import re

import pytest

from paper_1004_1680_gb300 import build as B
from paper_1004_1680_gb300 import mhd as M

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            text = open(os.path.join(ROOT, "include", h)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names += re.findall(r"\b(mhd_\w+)\s*\(", text)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return M.load()


def test_library_builds_for_sm103a(lib):
    assert os.path.exists(B.LIB)
    assert "arch=compute_103a,code=sm_103a" in " ".join(B.ARCH)


def test_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert "mhd_step" in names and "mhd_create" in names
    for n in names:
        assert hasattr(lib, n), n
    # and the binding covers them all
    assert set(names) <= set(M.SIGNATURES)


@pytest.mark.parametrize("dims,gamma", [((6, 4, 4), 5 / 3), ((0, 4, 4), 5 / 3), ((8, 0, 4), 5 / 3),
                                        ((8, 4, 4), 1.0), ((8, 4, 4), float("nan")),
                                        ((1 << 12, 1 << 10, 1 << 10), 5 / 3)])
def test_create_rejects_bad_arguments(lib, dims, gamma):
    assert not lib.mhd_create(dims[0], dims[1], dims[2], gamma)
    assert b"" != lib.mhd_last_error()


def test_null_handle_is_an_argument_error(lib):
    assert lib.mhd_step(None, 0.1) == M.MHD_E_ARG
    assert lib.mhd_run(None, 1, 0.7) == M.MHD_E_ARG
    assert lib.mhd_set_segments(None, 0, 0, 0) == M.MHD_E_ARG
    dt = ctypes.c_double()
    assert lib.mhd_cfl_dt(None, 0.7, ctypes.byref(dt)) == M.MHD_E_ARG
    lib.mhd_destroy(None)


@pytest.mark.parametrize("dims,cin,cout", [((12, 16, 4), 32, 32), ((8, 24, 4), 32, 32), ((8, 16, 0), 8, 32),
                                           ((8, 16, 4), 16, 32), ((8, 16, 4), 32, 64)])
def test_conv_rejects_unsupported_shapes(lib, dims, cin, cout):
    """Tiles are 8 x 16 x 1 cells and channels 8 or 32: anything else is an
    argument error, reported before any device work."""
    dummy = ctypes.c_void_p(16)
    nbytes = lib.mhd_conv_pack_bytes(cin, cout, 0)
    rc = lib.mhd_conv3d(dims[0], dims[1], dims[2], cin, cout, dummy, dummy, nbytes, None, 0, 0, None,
                        dummy, None, None)
    assert rc == M.MHD_E_ARG
    assert b"mhd_conv3d" in lib.mhd_last_error()


def test_conv_pack_sizes(lib):
    # 3 Npad rows (the three z taps side by side along N; Npad = 32 for 32
    # outputs, 16 for 8) x (9 in-plane offsets x cin, rounded up to 32) BF16
    assert lib.mhd_conv_pack_bytes(32, 32, 0) == 3 * 32 * 288 * 2
    assert lib.mhd_conv_pack_bytes(8, 32, 0) == 3 * 32 * 96 * 2
    assert lib.mhd_conv_pack_bytes(32, 8, 0) == 3 * 16 * 288 * 2
    assert lib.mhd_conv_pack_bytes(32, 8, 1) == 3 * 32 * 96 * 2
    assert lib.mhd_conv_pack_bytes(16, 8, 0) == 0


def test_submit_rejects_null_handle(lib):
    ptrs = (ctypes.c_void_p * 8)()
    assert lib.mhd_submit(None, ptrs, ptrs, 1, 0.7) == M.MHD_E_ARG
    assert lib.mhd_drain(None) == M.MHD_E_ARG


def test_set_scheme_rejects_null_handle(lib):
    assert lib.mhd_set_scheme(None, 0, 0) == M.MHD_E_ARG


def test_boundary_calls_reject_null_handle(lib):
    assert lib.mhd_set_boundary(None, 0, 1) == M.MHD_E_ARG
    assert lib.mhd_fill_ghosts(None) == M.MHD_E_ARG


def test_network_calls_reject_null_arguments(lib):
    nul4 = (ctypes.c_void_p * 4)()
    sz4 = (ctypes.c_size_t * 4)()
    nul3 = (ctypes.c_void_p * 3)()
    nul2 = (ctypes.c_void_p * 2)()
    assert lib.mhd_cnn_forward(8, 16, 2, None, nul4, sz4, nul4, nul3, None, None) == M.MHD_E_ARG
    assert lib.mhd_cnn_backward(8, 16, 2, None, nul3, None, nul4, sz4, nul4, nul4, nul2, None) == M.MHD_E_ARG
