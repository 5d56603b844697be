"""FP64 CPU oracle of the dimensionally split MHD grid update (test infrastructure).

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The CUDA library never does, and this
package imports nothing from it.

The arithmetic lives in ``mhd_oracle.c`` (plain loops, FP64, periodic
indexing, optional outflow or reflecting ghost layers); this module compiles it with gcc, loads it with ctypes and adds the
FP64 diagnostics (exactly rounded sums with ``math.fsum``) and the coarse-grid
restriction, both written from their plain definitions.  ``cnn.py`` is the
FP64 oracle of the learned coarse-grid correction (network, projection, loss,
clipped correction, Adam), with PyTorch CPU operations as library primitives.

State arrays are numpy float64 of shape (8, nz, ny, nx): fields rho, m_x, m_y,
m_z, e, b_x, b_y, b_z; b_d[k, j, i] lives on the low face of cell (i, j, k)
along d.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mhd_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lib = None
_lock = threading.Lock()

# -ffp-contract=off: no fused multiply-add, so x86 and Arm hosts give the
# same FP64 results; no -march flags for the same reason.
CFLAGS = ["-O2", "-std=c99", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off"]


def build(force: bool = False) -> str:
    """Compile mhd_oracle.c into _build/liboracle.so (if stale) and return its path."""
    os.makedirs(_BUILD, exist_ok=True)
    stale = (not os.path.exists(_LIB_PATH)
             or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC))
    if force or stale:
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", *CFLAGS, _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            dp = ctypes.POINTER(ctypes.c_double)
            i3 = ctypes.c_int * 3
            lib.orc_fluid_sweep.argtypes = [i3, ctypes.c_double, ctypes.c_void_p,
                                            ctypes.c_int, ctypes.c_double]
            lib.orc_mag_sweep.argtypes = [i3, ctypes.c_void_p, ctypes.c_int, ctypes.c_double]
            lib.orc_cfl_rate.argtypes = [i3, ctypes.c_double, ctypes.c_void_p]
            lib.orc_cfl_rate.restype = ctypes.c_double
            lib.orc_step.argtypes = [i3, ctypes.c_double, ctypes.c_void_p, ctypes.c_double]
            lib.orc_run.argtypes = [i3, ctypes.c_double, ctypes.c_void_p, ctypes.c_int,
                                    ctypes.c_double, dp]
            lib.orc_run.restype = ctypes.c_double
            lib.orc_threads.restype = ctypes.c_int
            lib.orc_set_threads.argtypes = [ctypes.c_int]
            lib.orc_set_pressure_floor.argtypes = [ctypes.c_double]
            lib.orc_set_resolution.argtypes = [ctypes.c_double] * 3
            lib.orc_set_scheme.argtypes = [ctypes.c_int, ctypes.c_int]
            lib.orc_set_scheme.restype = ctypes.c_int
            lib.orc_limiter.argtypes = [ctypes.c_double, ctypes.c_double]
            lib.orc_limiter.restype = ctypes.c_double
            lib.orc_freezing_speed.argtypes = [dp, dp, ctypes.c_double]
            lib.orc_freezing_speed.restype = ctypes.c_double
            lib.orc_set_boundary.argtypes = [ctypes.c_int, ctypes.c_int]
            lib.orc_set_boundary.restype = ctypes.c_int
            lib.orc_boundary.argtypes = [ctypes.c_int]
            lib.orc_boundary.restype = ctypes.c_int
            lib.orc_fill_ghosts.argtypes = [i3, ctypes.c_void_p]
            lib.orc_fill_ghosts.restype = ctypes.c_int
            _lib = lib
    return _lib


def _dims(state: np.ndarray):
    if state.dtype != np.float64 or state.ndim != 4 or state.shape[0] != 8:
        raise ValueError("state must be float64 of shape (8, nz, ny, nx)")
    if not state.flags.c_contiguous:
        raise ValueError("state must be C-contiguous")
    nz, ny, nx = state.shape[1:]
    return (ctypes.c_int * 3)(nx, ny, nz)


def _ptrs(state: np.ndarray):
    base = state.ctypes.data
    stride = state.strides[0]
    arr = (ctypes.c_void_p * 8)(*[base + q * stride for q in range(8)])
    return arr


def threads() -> int:
    """Number of OpenMP threads the oracle uses."""
    return _load().orc_threads()


def set_threads(t: int) -> None:
    _load().orc_set_threads(int(t))


def set_pressure_floor(p_floor: float) -> None:
    """Optional floor on the gas pressure after each fluid sweep (0 = off)."""
    _load().orc_set_pressure_floor(float(p_floor))


def set_resolution(cx: float = 0.0, cy: float = 0.0, cz: float = 0.0) -> None:
    """Cells per unit length along x, y, z (1/h; 0 = the box's own cell count,
    the periodic unit cube).  A slab of a larger periodic box keeps the whole
    box's h along the cut axis this way."""
    _load().orc_set_resolution(float(cx), float(cy), float(cz))


LIMITERS = {"vanleer": 0, "minmod": 1, "superbee": 2}
FREEZING = {"bound": 0, "fast": 1, "pencil": 2}


def set_scheme(limiter: str = "vanleer", freezing: str = "bound") -> None:
    """Scheme variant for the following sweeps (the paper's scheme is
    van Leer with the bound freezing speed; the others are ablations)."""
    if _load().orc_set_scheme(LIMITERS[limiter], FREEZING[freezing]):
        raise ValueError("bad scheme")


BOUNDARIES = {"periodic": 0, "outflow": 1, "reflecting": 2}
GHOST = 4  # ghost cells at each end of a non-periodic axis, inside the box


def set_boundary(axis: int, mode: str) -> None:
    """Boundary of axis (0=x, 1=y, 2=z) for the following sweeps: periodic
    (the paper's), outflow or reflecting (extensions; the axis then keeps
    GHOST ghost cells at each end, refilled before every sweep)."""
    if _load().orc_set_boundary(int(axis), BOUNDARIES[mode]):
        raise ValueError("bad boundary")


def boundary(axis: int) -> str:
    code = _load().orc_boundary(int(axis))
    return {v: k for k, v in BOUNDARIES.items()}[code]


class boundaries:
    """Context manager: boundaries(x="outflow", z="reflecting") sets the given
    axes and restores periodic boundaries on every axis at exit."""

    def __init__(self, **modes):
        self.modes = modes

    def __enter__(self):
        for name, mode in self.modes.items():
            set_boundary("xyz".index(name), mode)
        return self

    def __exit__(self, *exc):
        for a in range(3):
            set_boundary(a, "periodic")
        return False


def _check_boundary_dims(state: np.ndarray) -> None:
    nz, ny, nx = state.shape[1:]
    for a, n in enumerate((nx, ny, nz)):
        if _load().orc_boundary(a) and n < 3 * GHOST:
            raise ValueError(f"a non-periodic axis needs at least {3 * GHOST} cells")


def fill_ghosts(state: np.ndarray) -> None:
    """In place: refill the ghost layers of the non-periodic axes (the sweeps
    and the CFL rate do this themselves before they read the state)."""
    _check_boundary_dims(state)
    _load().orc_fill_ghosts(_dims(state), _ptrs(state))


def limiter(a: float, b: float) -> float:
    """phi(a, b) of the current limiter."""
    return _load().orc_limiter(float(a), float(b))


def freezing_speed(u, b, gamma: float) -> float:
    """Freezing speed of one cell, u = (rho, m_d, m_t1, m_t2, e), b = (b_d, b_t1, b_t2)."""
    ua = (ctypes.c_double * 5)(*[float(x) for x in u])
    ba = (ctypes.c_double * 3)(*[float(x) for x in b])
    return _load().orc_freezing_speed(ua, ba, float(gamma))


def fluid_sweep(state: np.ndarray, d: int, tau: float, gamma: float) -> None:
    """In place: relaxing-TVD fluid sweep along axis d (0=x, 1=y, 2=z), step tau."""
    _check_boundary_dims(state)
    _load().orc_fluid_sweep(_dims(state), gamma, _ptrs(state), int(d), float(tau))


def mag_sweep(state: np.ndarray, d: int, tau: float) -> None:
    """In place: magnetic advection-constraint sweep along axis d, step tau."""
    _check_boundary_dims(state)
    _load().orc_mag_sweep(_dims(state), _ptrs(state), int(d), float(tau))


def cfl_rate(state: np.ndarray, gamma: float) -> float:
    """max over cells and axes of (|v_d| + c_f*) / h_d."""
    _check_boundary_dims(state)
    return _load().orc_cfl_rate(_dims(state), gamma, _ptrs(state))


def cfl_dt(state: np.ndarray, gamma: float, cfl: float) -> float:
    """Full-step CFL timestep 2 * cfl / rate (each of the 6 sweeps uses dt/2)."""
    return 2.0 * cfl / cfl_rate(state, gamma)


def step(state: np.ndarray, dt: float, gamma: float) -> None:
    """In place: one full step (x, y, z then z, y, x; each sweep tau = dt/2)."""
    _check_boundary_dims(state)
    _load().orc_step(_dims(state), gamma, _ptrs(state), float(dt))


def run(state: np.ndarray, nsteps: int, cfl: float, gamma: float):
    """In place: nsteps full steps with per-step CFL dt. Returns (t, dts)."""
    _check_boundary_dims(state)
    dts = np.zeros(max(nsteps, 1), dtype=np.float64)
    t = _load().orc_run(_dims(state), gamma, _ptrs(state), int(nsteps), float(cfl),
                        dts.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    return t, dts[:nsteps]


# --------------------------------------------------------------------------
# FP64 diagnostics, from their plain definitions.

def diagnostics(state: np.ndarray, gamma: float) -> np.ndarray:
    """Ten numbers: exactly rounded sums of rho, m_x, m_y, m_z, e, b_x, b_y, b_z
    over all cells/faces; max over cells of |div b| * h_min; and the minimum
    gas pressure.

    div b of a cell is its discrete flux balance sum_d (b_d(high face) -
    b_d(low face)) / h_d (constrained transport keeps it at roundoff); it is
    multiplied by the smallest spacing h_min = 1/max(n) so it has the units of b.
    """
    _dims(state)
    nz, ny, nx = state.shape[1:]
    out = np.zeros(10, dtype=np.float64)
    for q in range(8):
        out[q] = math.fsum(state[q].ravel().tolist())
    n = (nx, ny, nz)
    div = np.zeros(state.shape[1:], dtype=np.float64)
    for d in range(3):
        b = state[5 + d]
        axis = 2 - d  # numpy axis of spatial axis d
        div += (np.roll(b, -1, axis=axis) - b) * n[d]
    out[8] = float(np.max(np.abs(div))) / max(n)
    out[9] = float(np.min(pressure(state, gamma)))
    return out


def pressure(state: np.ndarray, gamma: float) -> np.ndarray:
    """Gas pressure per cell, p = (gamma-1)(e - |m|^2/(2 rho) - |b_c|^2/2) (Eq. 3),
    b_c the mean of each cell's two faces."""
    rho = state[0]
    kin = 0.5 * (state[1] ** 2 + state[2] ** 2 + state[3] ** 2) / rho
    b2 = np.zeros_like(rho)
    for d in range(3):
        b = state[5 + d]
        bc = 0.5 * (b + np.roll(b, -1, axis=2 - d))
        b2 += bc * bc
    return (gamma - 1.0) * (state[4] - kin - 0.5 * b2)


def restrict(state: np.ndarray, r: int) -> np.ndarray:
    """Coarse-grid restriction by an integer factor r along every axis.

    Conserved cell quantities: mean over the r^3 fine cells of a coarse cell.
    Face field b_d: mean over the r^2 fine faces that tile the coarse face
    (the fine faces at fine index r*I along d).  The coarse face flux equals
    the sum of the fine fluxes, so a divergence-free fine field restricts to a
    divergence-free coarse field.
    """
    _dims(state)
    nz, ny, nx = state.shape[1:]
    if nx % r or ny % r or nz % r:
        raise ValueError("dims must be divisible by r")
    Z, Y, X = nz // r, ny // r, nx // r
    out = np.empty((8, Z, Y, X), dtype=np.float64)
    for q in range(5):
        out[q] = state[q].reshape(Z, r, Y, r, X, r).mean(axis=(1, 3, 5))
    bx = state[5][:, :, ::r]                      # faces on coarse x-faces
    out[5] = bx.reshape(Z, r, Y, r, X).mean(axis=(1, 3))
    by = state[6][:, ::r, :]
    out[6] = by.reshape(Z, r, Y, X, r).mean(axis=(1, 4))
    bz = state[7][::r, :, :]
    out[7] = bz.reshape(Z, Y, r, X, r).mean(axis=(2, 4))
    return out
