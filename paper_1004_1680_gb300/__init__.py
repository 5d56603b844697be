"""GB300-native dimensionally split ideal-MHD grid update (relaxing-TVD fluid
sweeps + constrained-transport magnetic sweeps, x-y-z then z-y-x) of Pang, Pen
& Perrone, "Magnetohydrodynamics on Heterogeneous architectures".

The compute path is the CUDA library built from csrc/ (C ABI in include/mhd.h);
``mhd`` is its Python binding and ``initial_conditions`` builds seeded inputs.
"""
from . import build  # noqa: F401

__all__ = ["build", "mhd", "initial_conditions"]
