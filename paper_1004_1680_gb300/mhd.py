"""Python binding of the C ABI in include/mhd.h (argument marshalling only).

Every step of the update runs in the CUDA library libmhd_gb300.so; this module
only converts torch tensors / numpy arrays into pointers and return codes
into exceptions.  There is no fallback: if the library or a GPU is missing,
constructing a Box raises.

State tensors have shape (8, nz, ny, nx), dtype float32, fields in the order
rho, m_x, m_y, m_z, e, b_x, b_y, b_z (b_d on the low face of each cell).
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np
import torch

from . import build as _build

MHD_OK, MHD_E_ARG, MHD_E_CUDA, MHD_E_OOM, MHD_E_STATE, MHD_E_TIMEOUT = range(6)
_ERR_NAMES = {1: "MHD_E_ARG", 2: "MHD_E_CUDA", 3: "MHD_E_OOM", 4: "MHD_E_STATE", 5: "MHD_E_TIMEOUT"}

_lib = None
_lock = threading.Lock()

# Exported symbols and their ctypes signatures (kept in sync with include/mhd.h).
_P = ctypes.c_void_p
_I = ctypes.c_int
_D = ctypes.c_double
_PP = ctypes.POINTER(ctypes.c_void_p)
_DP = ctypes.POINTER(ctypes.c_double)
SIGNATURES = {
    "mhd_create": (_P, [_I, _I, _I, _D]),
    "mhd_destroy": (None, [_P]),
    "mhd_set_stream": (_I, [_P, _P]),
    "mhd_set_state": (_I, [_P, _PP, _I]),
    "mhd_get_state": (_I, [_P, _PP, _I]),
    "mhd_cfl_dt": (_I, [_P, _D, _DP]),
    "mhd_step": (_I, [_P, _D]),
    "mhd_run": (_I, [_P, _I, _D]),
    "mhd_submit": (_I, [_P, _PP, _PP, _I, _D]),
    "mhd_drain": (_I, [_P]),
    "mhd_time": (_I, [_P, _DP]),
    "mhd_sweep": (_I, [_P, _I, _I, _D]),
    "mhd_set_segments": (_I, [_P, _I, _I, _I]),
    "mhd_set_xpath": (_I, [_P, _I]),
    "mhd_set_fusion": (_I, [_P, _I]),
    "mhd_set_tma": (_I, [_P, _I]),
    "mhd_tma_sweeps": (_I, [_P, ctypes.POINTER(ctypes.c_longlong)]),
    "mhd_create_f64": (_P, [_I, _I, _I, _D]),
    "mhd_set_state_f64": (_I, [_P, _PP, _I]),
    "mhd_get_state_f64": (_I, [_P, _PP, _I]),
    "mhd_set_resolution": (_I, [_P, _D, _D, _D]),
    "mhd_set_interior": (_I, [_P, _I, _I, _I]),
    "mhd_copy_planes": (_I, [_P, _I, _I, _PP, _I, _I]),
    "mhd_set_pressure_floor": (_I, [_P, _D]),
    "mhd_set_scheme": (_I, [_P, _I, _I]),
    "mhd_set_boundary": (_I, [_P, _I, _I]),
    "mhd_fill_ghosts": (_I, [_P]),
    "mhd_ens_set_pressure_floor": (_I, [_P, _D]),
    "mhd_diagnostics": (_I, [_P, _DP]),
    "mhd_profile": (_I, [_P, _I]),
    "mhd_profile_read": (_I, [_P, ctypes.POINTER(ctypes.c_int), _DP]),
    "mhd_diagnostics_static": (_I, [_I, _I, _I, _D, _PP, _DP, _P]),
    "mhd_ens_create": (_P, [_I, ctypes.POINTER(ctypes.c_int), _D]),
    "mhd_ens_destroy": (None, [_P]),
    "mhd_ens_set_stream": (_I, [_P, _P]),
    "mhd_ens_set_state": (_I, [_P, _I, _PP, _I]),
    "mhd_ens_get_state": (_I, [_P, _I, _PP, _I]),
    "mhd_ens_run": (_I, [_P, _I, _D]),
    "mhd_ens_times": (_I, [_P, _DP]),
    "mhd_ens_cfl_dt": (_I, [_P, _D, _DP]),
    "mhd_ens_diagnostics": (_I, [_P, _DP]),
    "mhd_ens_set_tuning": (_I, [_P, _I, _I]),
    "mhd_ens_autotune": (_I, [_P, _D, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
    "mhd_conv_pack_bytes": (ctypes.c_size_t, [_I, _I, _I]),
    "mhd_conv_pack": (_I, [_P, _I, _I, _I, _P, _P]),
    "mhd_conv3d": (_I, [_I, _I, _I, _I, _I, _P, _P, ctypes.c_size_t, _P, _I, _I, _P, _P, _P, _P]),
    "mhd_conv3d_wgrad": (_I, [_I, _I, _I, _I, _I, _P, _P, _P, _P, _P]),
    "mhd_cnn_forward": (_I, [_I, _I, _I, _P, _PP, ctypes.POINTER(ctypes.c_size_t), _PP, _PP, _P, _P]),
    "mhd_cnn_backward": (_I, [_I, _I, _I, _P, _PP, _P, _PP, ctypes.POINTER(ctypes.c_size_t), _PP, _PP, _PP,
                              _P]),
    "mhd_conv_error": (_I, [ctypes.POINTER(ctypes.c_int)]),
    "mhd_restrict": (_I, [_I, _I, _I, _I, _PP, _PP, _P]),
    "mhd_cnn_normalize": (_I, [_I, _I, _I, _PP, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_float),
                               _P, _P]),
    "mhd_cnn_project": (_I, [_I, _I, _I, _P, ctypes.POINTER(ctypes.c_float), _PP, _P, _P]),
    "mhd_cnn_loss": (_I, [_I, _I, _I, _PP, _PP, ctypes.POINTER(ctypes.c_float), _P, _PP, _P]),
    "mhd_cnn_project_backward": (_I, [_I, _I, _I, _PP, ctypes.POINTER(ctypes.c_float), _P, _P, _P]),
    "mhd_correct": (_I, [_I, _I, _I, _PP, _PP, _P, _P, _P]),
    "mhd_adam": (_I, [_P, _P, _P, _P, _I, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float, _I,
                      _P]),
    "mhd_last_error": (ctypes.c_char_p, []),
}


KERNEL_CLASSES = ["fluid_x", "fluid_y", "fluid_z", "mag_x", "mag_y", "mag_z", "control", "transpose"]
K_CLASSES = len(KERNEL_CLASSES)


class MHDError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_ERR_NAMES.get(code, code)}: {msg}")
        self.code = code


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True) -> ctypes.CDLL:
    """Load libmhd_gb300.so (building it first if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.LIB
            if build_if_missing and _build.stale():
                _build.build()
            if not os.path.exists(path):
                raise RuntimeError(f"CUDA library not built: {path}")
            lib = ctypes.CDLL(path)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def _check(rc: int):
    if rc != MHD_OK:
        raise MHDError(rc, _lib.mhd_last_error().decode())


def _field_ptrs(t: torch.Tensor):
    return (ctypes.c_void_p * 8)(*[t[q].data_ptr() for q in range(8)])


def diagnostics_static(state: torch.Tensor, gamma: float = 5.0 / 3.0, stream=None) -> np.ndarray:
    """FP64 diagnostics of a float32 CUDA state tensor (8, nz, ny, nx) through
    mhd_diagnostics_static: no mhd_t and no device allocation."""
    lib = load()
    if not state.is_cuda or state.dtype != torch.float32 or not state.is_contiguous():
        raise ValueError("state must be a contiguous float32 CUDA tensor")
    nz, ny, nx = state.shape[1:]
    s = stream if stream is not None else torch.cuda.current_stream()
    out = (ctypes.c_double * 10)()
    _check(lib.mhd_diagnostics_static(nx, ny, nz, gamma, _field_ptrs(state), out,
                                      ctypes.c_void_p(s.cuda_stream)))
    return np.array(out[:], dtype=np.float64)


class Box:
    """One periodic MHD box on the current CUDA device (wraps mhd_t)."""

    def __init__(self, nx: int, ny: int, nz: int, gamma: float = 5.0 / 3.0, stream=None):
        if not torch.cuda.is_available():
            raise RuntimeError("a CUDA GPU is required (no CPU fallback)")
        self.lib = load()
        self.shape = (8, nz, ny, nx)
        self.n = (nx, ny, nz)
        self.gamma = gamma
        h = self.lib.mhd_create(nx, ny, nz, gamma)
        if not h:
            raise MHDError(MHD_E_ARG, self.lib.mhd_last_error().decode())
        self.h = ctypes.c_void_p(h)
        self.set_stream(stream if stream is not None else torch.cuda.current_stream())

    def close(self):
        if getattr(self, "h", None):
            self.lib.mhd_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_stream(self, stream):
        ptr = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
        self.stream = stream
        _check(self.lib.mhd_set_stream(self.h, ctypes.c_void_p(ptr)))

    def set_state(self, state: torch.Tensor):
        """Copy a float32 (8, nz, ny, nx) state in (CUDA or host tensor)."""
        if state.shape != self.shape or state.dtype != torch.float32 or not state.is_contiguous():
            raise ValueError(f"state must be contiguous float32 {self.shape}")
        _check(self.lib.mhd_set_state(self.h, _field_ptrs(state), 1 if state.is_cuda else 0))
        self._keep = state  # the copy is asynchronous: keep the source alive

    def get_state(self, out: torch.Tensor | None = None, device="cuda") -> torch.Tensor:
        if out is None:
            out = torch.empty(self.shape, dtype=torch.float32, device=device)
        if out.shape != self.shape or out.dtype != torch.float32 or not out.is_contiguous():
            raise ValueError("bad output tensor")
        _check(self.lib.mhd_get_state(self.h, _field_ptrs(out), 1 if out.is_cuda else 0))
        return out

    def submit(self, state_in: torch.Tensor, state_out: torch.Tensor, nsteps: int = 1, cfl: float = 0.7):
        """Pipelined host run: copy the host state in, run nsteps (device CFL),
        copy the result into the host tensor state_out; returns at once (see
        drain).  Both tensors: contiguous float32 (8, nz, ny, nx), pinned."""
        for t in (state_in, state_out):
            if t.shape != self.shape or t.dtype != torch.float32 or not t.is_contiguous() or t.is_cuda:
                raise ValueError(f"host state must be contiguous float32 {self.shape}")
        _check(self.lib.mhd_submit(self.h, _field_ptrs(state_in), _field_ptrs(state_out), int(nsteps), float(cfl)))
        self._pending = getattr(self, "_pending", []) + [(state_in, state_out)]

    def drain(self):
        """Wait until every submitted run's result is in its host tensor."""
        _check(self.lib.mhd_drain(self.h))
        self._pending = []

    def cfl_dt(self, cfl: float = 0.7) -> float:
        dt = ctypes.c_double()
        _check(self.lib.mhd_cfl_dt(self.h, cfl, ctypes.byref(dt)))
        return dt.value

    def step(self, dt: float):
        _check(self.lib.mhd_step(self.h, float(dt)))

    def run(self, nsteps: int, cfl: float = 0.7):
        _check(self.lib.mhd_run(self.h, int(nsteps), float(cfl)))

    def time(self) -> float:
        t = ctypes.c_double()
        _check(self.lib.mhd_time(self.h, ctypes.byref(t)))
        return t.value

    def sweep(self, axis: int, kind: int, tau: float):
        """kind 0: fluid sweep, kind 1: magnetic sweep, along axis with step tau."""
        _check(self.lib.mhd_sweep(self.h, int(axis), int(kind), float(tau)))

    def set_segments(self, sx: int = 0, sy: int = 0, sz: int = 0):
        _check(self.lib.mhd_set_segments(self.h, int(sx), int(sy), int(sz)))

    def set_pressure_floor(self, p_floor: float):
        """Optional floor on the gas pressure after fluid sweeps (0 = off)."""
        _check(self.lib.mhd_set_pressure_floor(self.h, float(p_floor)))

    LIMITERS = {"vanleer": 0, "minmod": 1, "superbee": 2}
    FREEZING = {"bound": 0, "fast": 1, "pencil": 2}

    def set_scheme(self, limiter: str = "vanleer", freezing: str = "bound"):
        """Scheme variant (ablation) for the following sweeps; the default is
        the paper's scheme."""
        _check(self.lib.mhd_set_scheme(self.h, self.LIMITERS[limiter], self.FREEZING[freezing]))

    BOUNDARIES = {"periodic": 0, "outflow": 1, "reflecting": 2}
    GHOST = 4

    def set_boundary(self, axis: int, mode: str):
        """Boundary of physical axis 0/1/2: periodic (the paper's), outflow or
        reflecting; a non-periodic axis keeps GHOST ghost cells at each end
        inside the box (at least 12 cells in all), refilled before every sweep."""
        _check(self.lib.mhd_set_boundary(self.h, int(axis), self.BOUNDARIES[mode]))

    def fill_ghosts(self):
        """Refill the ghost layers of the non-periodic axes now."""
        _check(self.lib.mhd_fill_ghosts(self.h))

    def set_resolution(self, cx: float = 0.0, cy: float = 0.0, cz: float = 0.0):
        """Cells per unit length along x, y, z (1/h; 0 = the box's own cell
        count, the unit box)."""
        _check(self.lib.mhd_set_resolution(self.h, float(cx), float(cy), float(cz)))

    def set_interior(self, axis: int, lo: int, hi: int):
        """Cells [lo, hi) along axis are this box's own (the CFL rate covers
        them only); the rest are halo copies."""
        _check(self.lib.mhd_set_interior(self.h, int(axis), int(lo), int(hi)))

    def get_planes(self, z0: int, nplanes: int, out: torch.Tensor | None = None) -> torch.Tensor:
        """z-planes z0 .. z0+nplanes-1 of the 8 fields as a (8, nplanes, ny, nx)
        float32 CUDA tensor (stream ordered)."""
        nx, ny, nz = self.n
        if out is None:
            out = torch.empty((8, nplanes, ny, nx), dtype=torch.float32, device="cuda")
        _check(self.lib.mhd_copy_planes(self.h, int(z0), int(nplanes), _field_ptrs(out), 0, 1))
        return out

    def set_planes(self, z0: int, planes: torch.Tensor):
        """Write a (8, nplanes, ny, nx) float32 CUDA tensor into z-planes
        z0 .. z0+nplanes-1 (stream ordered)."""
        if not planes.is_cuda or planes.dtype != torch.float32 or not planes.is_contiguous():
            raise ValueError("planes must be a contiguous float32 CUDA tensor")
        _check(self.lib.mhd_copy_planes(self.h, int(z0), int(planes.shape[1]), _field_ptrs(planes), 1, 1))

    def set_fusion(self, on: bool):
        """Run the two middle z magnetic sweeps of a step as one launch (on,
        the default) or as two (off); the state is bitwise the same."""
        _check(self.lib.mhd_set_fusion(self.h, int(bool(on))))

    def set_tma(self, on: bool):
        """Stage the y and z kernel-axis sweeps' input with TMA tile copies
        where the box qualifies (on, the default) or use register loads
        (off); the two agree to FP32 rounding (the staged fluid sweep takes
        the hardware square root approximation)."""
        _check(self.lib.mhd_set_tma(self.h, int(bool(on))))

    def tma_sweeps(self) -> int:
        """Sweeps (fluid and magnetic) this box has launched TMA-staged so far."""
        n = ctypes.c_longlong(0)
        _check(self.lib.mhd_tma_sweeps(self.h, ctypes.byref(n)))
        return int(n.value)

    def set_xpath(self, mode: int):
        """x sweeps: 1 direct, 2 through the x<->y exchanged layout, 0 automatic;
        3: every sweep along the contiguous axis of a transposed copy (the
        paper's data flow, an ablation)."""
        _check(self.lib.mhd_set_xpath(self.h, int(mode)))

    def profile(self, capacity: int):
        """Time every later kernel launch with CUDA events (up to `capacity`)."""
        _check(self.lib.mhd_profile(self.h, int(capacity)))

    def profile_read(self) -> dict:
        """{kernel class: (launches, total device ms)} since profile()."""
        c = (ctypes.c_int * K_CLASSES)()
        t = (ctypes.c_double * K_CLASSES)()
        _check(self.lib.mhd_profile_read(self.h, c, t))
        return {KERNEL_CLASSES[k]: (c[k], t[k]) for k in range(K_CLASSES)}

    def diagnostics(self) -> np.ndarray:
        out = (ctypes.c_double * 10)()
        _check(self.lib.mhd_diagnostics(self.h, out))
        return np.array(out[:], dtype=np.float64)


class Box64:
    """One periodic box computed in FP64 on the GPU (wraps an mhd_t made by
    mhd_create_f64): the paper's scheme in double precision, an ablation of
    the FP32 path."""

    def __init__(self, nx: int, ny: int, nz: int, gamma: float = 5.0 / 3.0, stream=None):
        if not torch.cuda.is_available():
            raise RuntimeError("a CUDA GPU is required (no CPU fallback)")
        self.lib = load()
        self.shape = (8, nz, ny, nx)
        self.n = (nx, ny, nz)
        self.gamma = gamma
        h = self.lib.mhd_create_f64(nx, ny, nz, gamma)
        if not h:
            raise MHDError(MHD_E_ARG, self.lib.mhd_last_error().decode())
        self.h = ctypes.c_void_p(h)
        s = stream if stream is not None else torch.cuda.current_stream()
        _check(self.lib.mhd_set_stream(self.h, ctypes.c_void_p(s.cuda_stream)))

    def close(self):
        if getattr(self, "h", None):
            self.lib.mhd_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_state(self, state: torch.Tensor):
        if state.shape != self.shape or state.dtype != torch.float64 or not state.is_contiguous():
            raise ValueError("state must be a contiguous float64 tensor (8, nz, ny, nx)")
        _check(self.lib.mhd_set_state_f64(self.h, _field_ptrs(state), 1 if state.is_cuda else 0))
        if not state.is_cuda:
            torch.cuda.synchronize()

    def get_state(self, device="cuda") -> torch.Tensor:
        out = torch.empty(self.shape, dtype=torch.float64, device=device)
        _check(self.lib.mhd_get_state_f64(self.h, _field_ptrs(out), 1 if out.is_cuda else 0))
        return out

    def cfl_dt(self, cfl: float = 0.7) -> float:
        dt = ctypes.c_double()
        _check(self.lib.mhd_cfl_dt(self.h, cfl, ctypes.byref(dt)))
        return dt.value

    def step(self, dt: float):
        _check(self.lib.mhd_step(self.h, float(dt)))

    def run(self, nsteps: int, cfl: float = 0.7):
        _check(self.lib.mhd_run(self.h, int(nsteps), float(cfl)))

    def sweep(self, axis: int, kind: int, tau: float):
        _check(self.lib.mhd_sweep(self.h, int(axis), int(kind), float(tau)))

    def time(self) -> float:
        t = ctypes.c_double()
        _check(self.lib.mhd_time(self.h, ctypes.byref(t)))
        return t.value


class Ensemble:
    """Many independent periodic boxes advanced together (wraps mhd_ens_t)."""

    def __init__(self, dims, gamma: float = 5.0 / 3.0, stream=None):
        if not torch.cuda.is_available():
            raise RuntimeError("a CUDA GPU is required (no CPU fallback)")
        self.lib = load()
        self.dims = [tuple(int(v) for v in d) for d in dims]
        self.gamma = gamma
        flat = (ctypes.c_int * (3 * len(self.dims)))(*[v for d in self.dims for v in d])
        h = self.lib.mhd_ens_create(len(self.dims), flat, gamma)
        if not h:
            raise MHDError(MHD_E_ARG, self.lib.mhd_last_error().decode())
        self.h = ctypes.c_void_p(h)
        s = stream if stream is not None else torch.cuda.current_stream()
        self.stream = s
        _check(self.lib.mhd_ens_set_stream(self.h, ctypes.c_void_p(s.cuda_stream)))
        self._keep = {}

    def close(self):
        if getattr(self, "h", None):
            self.lib.mhd_ens_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def shape(self, b):
        nx, ny, nz = self.dims[b]
        return (8, nz, ny, nx)

    def set_state(self, b: int, state: torch.Tensor):
        if state.shape != self.shape(b) or state.dtype != torch.float32 or not state.is_contiguous():
            raise ValueError(f"state must be contiguous float32 {self.shape(b)}")
        _check(self.lib.mhd_ens_set_state(self.h, int(b), _field_ptrs(state), 1 if state.is_cuda else 0))
        self._keep[b] = state

    def get_state(self, b: int, device="cuda") -> torch.Tensor:
        out = torch.empty(self.shape(b), dtype=torch.float32, device=device)
        _check(self.lib.mhd_ens_get_state(self.h, int(b), _field_ptrs(out), 1 if out.is_cuda else 0))
        return out

    def run(self, nsteps: int, cfl: float = 0.7):
        _check(self.lib.mhd_ens_run(self.h, int(nsteps), float(cfl)))

    def times(self) -> np.ndarray:
        out = (ctypes.c_double * len(self.dims))()
        _check(self.lib.mhd_ens_times(self.h, out))
        return np.array(out[:])

    def cfl_dt(self, cfl: float = 0.7) -> np.ndarray:
        out = (ctypes.c_double * len(self.dims))()
        _check(self.lib.mhd_ens_cfl_dt(self.h, cfl, out))
        return np.array(out[:])

    def cfl_dt_safe(self, cfl: float = 0.7) -> np.ndarray:
        """Like cfl_dt, but invalid boxes give 0 instead of raising."""
        out = (ctypes.c_double * len(self.dims))()
        rc = self.lib.mhd_ens_cfl_dt(self.h, cfl, out)
        if rc not in (MHD_OK, MHD_E_STATE):
            _check(rc)
        return np.array(out[:])

    def diagnostics(self) -> np.ndarray:
        out = (ctypes.c_double * (10 * len(self.dims)))()
        _check(self.lib.mhd_ens_diagnostics(self.h, out))
        return np.array(out[:]).reshape(len(self.dims), 10)

    def set_pressure_floor(self, p_floor: float):
        _check(self.lib.mhd_ens_set_pressure_floor(self.h, float(p_floor)))

    def set_tuning(self, xpath: int, segdiv: int):
        _check(self.lib.mhd_ens_set_tuning(self.h, int(xpath), int(segdiv)))

    def autotune(self, cfl: float = 0.7):
        x, s = ctypes.c_int(), ctypes.c_int()
        _check(self.lib.mhd_ens_autotune(self.h, cfl, ctypes.byref(x), ctypes.byref(s)))
        return x.value, s.value


# --------------------------------------------------------------------------
# tensor-core 3-D convolution (learned correction)

def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def conv_pack(w: torch.Tensor, transpose: bool = False, stream=None) -> torch.Tensor:
    """Pack FP32 weights (cout, cin, 3, 3, 3) into the BF16 tensor-core image."""
    lib = load()
    cout, cin = w.shape[:2]
    nbytes = lib.mhd_conv_pack_bytes(cin, cout, int(transpose))
    img = torch.empty(nbytes // 2, dtype=torch.int16, device=w.device)
    _check(lib.mhd_conv_pack(_ptr(w.contiguous()), cin, cout, int(transpose), _ptr(img), _stream(stream)))
    return img


def conv3d(x: torch.Tensor, img: torch.Tensor, n, cin: int, cout: int, bias=None, relu=False, flip=False,
           mask=None, out_bf16=True, out_f32=False, stream=None):
    """Periodic 3x3x3 convolution of channels-last BF16 x (cells, cin).
    Returns (y_bf16 or None, y_f32 or None), each (cells, cout)."""
    lib = load()
    cells = n[0] * n[1] * n[2]
    yb = torch.empty((cells, cout), dtype=torch.bfloat16, device=x.device) if out_bf16 else None
    yf = torch.empty((cells, cout), dtype=torch.float32, device=x.device) if out_f32 else None
    _check(lib.mhd_conv3d(n[0], n[1], n[2], cin, cout, _ptr(x), _ptr(img), img.numel() * img.element_size(),
                          _ptr(bias), int(relu), int(flip), _ptr(mask), _ptr(yb), _ptr(yf), _stream(stream)))
    return yb, yf


def conv3d_into(x: torch.Tensor, img: torch.Tensor, n, cin: int, cout: int, y_bf16=None, y_f32=None, bias=None,
                relu=False, flip=False, mask=None, stream=None):
    """conv3d writing into caller-provided outputs (no allocation)."""
    lib = load()
    _check(lib.mhd_conv3d(n[0], n[1], n[2], cin, cout, _ptr(x), _ptr(img), img.numel() * img.element_size(),
                          _ptr(bias), int(relu), int(flip), _ptr(mask), _ptr(y_bf16), _ptr(y_f32), _stream(stream)))


def conv3d_wgrad(x: torch.Tensor, gy: torch.Tensor, n, cin: int, cout: int, gw: torch.Tensor, gb=None,
                 stream=None):
    """Accumulate the weight (and bias) gradient into gw (cout*cin*27) and gb."""
    lib = load()
    _check(lib.mhd_conv3d_wgrad(n[0], n[1], n[2], cin, cout, _ptr(x), _ptr(gy), _ptr(gw), _ptr(gb),
                                _stream(stream)))


def _ptr_array(ts):
    return (ctypes.c_void_p * len(ts))(*[_ptr(t) for t in ts])


def _bytes_array(ts):
    return (ctypes.c_size_t * len(ts))(*[t.numel() * t.element_size() for t in ts])


def cnn_forward(x: torch.Tensor, imgs, biases, acts, y: torch.Tensor, n, stream=None):
    """The 4-layer correction network in one call (mhd_cnn_forward): x (cells, 8)
    BF16 -> y (cells, 8) FP32; acts: three (cells, 32) BF16 buffers that
    receive the hidden activations."""
    lib = load()
    _check(lib.mhd_cnn_forward(n[0], n[1], n[2], _ptr(x), _ptr_array(imgs), _bytes_array(imgs),
                               _ptr_array(biases), _ptr_array(acts), _ptr(y), _stream(stream)))


def cnn_backward(x: torch.Tensor, acts, gy: torch.Tensor, imgsT, gws, gbs, scratch, n, stream=None):
    """Backward of cnn_forward for gy (cells, 8) BF16 (mhd_cnn_backward):
    accumulates the weight and bias gradients into gws / gbs."""
    lib = load()
    _check(lib.mhd_cnn_backward(n[0], n[1], n[2], _ptr(x), _ptr_array(acts), _ptr(gy), _ptr_array(imgsT),
                                _bytes_array(imgsT), _ptr_array(gws), _ptr_array(gbs), _ptr_array(scratch),
                                _stream(stream)))


def conv_error() -> int:
    lib = load()
    f = ctypes.c_int()
    rc = lib.mhd_conv_error(ctypes.byref(f))
    if rc not in (MHD_OK, MHD_E_TIMEOUT):
        _check(rc)
    return f.value


def _fields(t):
    """8 field pointers of an (8, ...) tensor (None -> null array)."""
    if t is None:
        return ctypes.cast(0, _PP)
    return _field_ptrs(t)


def _floats(v):
    v = [float(x) for x in v]
    return (ctypes.c_float * len(v))(*v)


def restrict(fine: torch.Tensor, r: int, stream=None) -> torch.Tensor:
    """Restrict an (8, nz, ny, nx) FP32 CUDA state by r along every axis."""
    lib = load()
    nz, ny, nx = fine.shape[1:]
    out = torch.empty((8, nz // r, ny // r, nx // r), dtype=torch.float32, device=fine.device)
    _check(lib.mhd_restrict(nx, ny, nz, r, _fields(fine), _fields(out), _stream(stream)))
    return out


def cnn_normalize(state, mu, inv_sigma, out=None, stream=None):
    lib = load()
    nz, ny, nx = state.shape[1:]
    if out is None:
        out = torch.empty((nx * ny * nz, 8), dtype=torch.bfloat16, device=state.device)
    _check(lib.mhd_cnn_normalize(nx, ny, nz, _fields(state), _floats(mu), _floats(inv_sigma), _ptr(out),
                                 _stream(stream)))
    return out


def cnn_project(y, n, scale, out=None, sums=None, stream=None):
    lib = load()
    nx, ny, nz = n
    if out is None:
        out = torch.empty((8, nz, ny, nx), dtype=torch.float32, device=y.device)
    if sums is None:
        sums = torch.empty(5, dtype=torch.float64, device=y.device)
    _check(lib.mhd_cnn_project(nx, ny, nz, _ptr(y), _floats(scale), _fields(out), _ptr(sums), _stream(stream)))
    return out


def cnn_loss(d, t, weight, g=None, loss=None, stream=None):
    lib = load()
    nz, ny, nx = d.shape[1:]
    if loss is None:
        loss = torch.empty(1, dtype=torch.float64, device=d.device)
    _check(lib.mhd_cnn_loss(nx, ny, nz, _fields(d), _fields(t), _floats(weight), _ptr(loss), _fields(g),
                            _stream(stream)))
    return loss


def cnn_project_backward(g, scale, out=None, sums=None, stream=None):
    lib = load()
    nz, ny, nx = g.shape[1:]
    if out is None:
        out = torch.empty((nx * ny * nz, 8), dtype=torch.bfloat16, device=g.device)
    if sums is None:
        sums = torch.empty(5, dtype=torch.float64, device=g.device)
    _check(lib.mhd_cnn_project_backward(nx, ny, nz, _fields(g), _floats(scale), _ptr(sums), _ptr(out),
                                        _stream(stream)))
    return out


def correct(state, d, scratch=None, nclip=None, stream=None):
    lib = load()
    nz, ny, nx = state.shape[1:]
    if scratch is None:
        scratch = torch.empty(nx * ny * nz, dtype=torch.float32, device=state.device)
    _check(lib.mhd_correct(nx, ny, nz, _fields(state), _fields(d), _ptr(scratch), _ptr(nclip), _stream(stream)))


def adam(p, g, m, v, lr, step, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
    lib = load()
    _check(lib.mhd_adam(_ptr(p), _ptr(g), _ptr(m), _ptr(v), p.numel(), lr, beta1, beta2, eps, int(step),
                        _stream(stream)))
