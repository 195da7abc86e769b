"""CPU oracle (FP64, numpy) of the staggered FFT non-local damage scheme.

TEST INFRASTRUCTURE ONLY: imported by the test suite, the smoke check and the
benchmark's CPU-baseline leg; never by the product path.  It shares no code
with the CUDA library.
"""
from .rve_oracle import *  # noqa: F401,F403
from . import rve_oracle  # noqa: F401
