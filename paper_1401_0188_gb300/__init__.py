"""GB300 (sm_103a) D2Q13 energy-conserving MRT lattice Boltzmann time step.

The compute path is the CUDA library built from csrc/ (C ABI in
include/lbm13.h); this package is its ctypes binding plus host-side helpers.
"""
from .params import pstar, rest_temperature  # noqa: F401
from .lbm13 import Lattice  # noqa: F401

__all__ = ["pstar", "rest_temperature", "Lattice"]
