"""GB300 (sm_103a) implementation of the per-time-step lattice update of the improved 3D
thermal pseudopotential lattice Boltzmann model (Li, Yu & Luo, arXiv 2201.06039).

The product is the C-ABI library built from csrc/ (include/lbm.h); `lbm` is its thin
ctypes binding, `thermo` the host-side Peng-Robinson helpers used to set up initial fields.
"""
from .lbm import *  # noqa: F401,F403
from . import lbm, thermo  # noqa: F401
