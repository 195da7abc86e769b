"""GB300 library for non-local ductile damage in voxelised periodic RVEs:
the hot path of the staggered FFT scheme (return map, FFT-Galerkin mechanics
under mixed control, preconditioned Helmholtz solve) as sm_103a CUDA kernels
behind the C ABI of include/rve.h, with this ctypes binding on top."""
from ._binding import *  # noqa: F401,F403
from ._binding import lib, RVE, RVEError  # noqa: F401
