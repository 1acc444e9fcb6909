"""GB300-native reduced-order Newton / FETI-DP solver for neo-Hookean lattice structures.

The compute path is liblattice.so (hand-written CUDA for sm_103a, C ABI in include/lattice.h);
``lattice`` is its ctypes binding and ``solver`` the load-stepping / autograd wrapper.
"""
from .lattice import (LAT_FP64, LAT_MIXED_BF16, LAT_MIXED_FP32, Lattice, LatticeError, NewtonOpts,
                      NewtonReport, case_arrays, load_library)
from .solver import Compliance, solve_load_path

__all__ = ["Lattice", "LatticeError", "NewtonOpts", "NewtonReport", "case_arrays", "load_library",
           "solve_load_path", "Compliance", "LAT_FP64", "LAT_MIXED_FP32", "LAT_MIXED_BF16"]
