"""Plain FP64 CPU oracle of the maximum-likelihood map-making solve (test infrastructure only).

This package is the independent checker for the CUDA path.  Only the test-suite, the smoke entry
point and the CPU-baseline leg of the benchmark may import it; the library never does.  It shares
no code with the CUDA path.

See :mod:`oracle.mapmaking` for the functions and the paper passages each follows.
"""
from .mapmaking import *  # noqa: F401,F403
