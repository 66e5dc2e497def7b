"""GB300-native staggered-leapfrog lattice evolution of two interacting scalar
fields in an expanding FRW universe (after Sainio, arXiv:0911.5692).

The compute path is the CUDA library built from csrc/ (C ABI in
include/lattice.h); this package holds its Python binding and the workload
presets.
"""
from .lattice import EXPORTED, Ensemble, Lattice, LatticeError, load_library, library_path, make_params  # noqa: F401
from . import workloads  # noqa: F401

__all__ = ["Ensemble", "Lattice", "LatticeError", "load_library", "library_path", "make_params", "workloads", "EXPORTED"]
