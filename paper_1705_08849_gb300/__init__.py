"""GB300-native (sm_103a) matrix-free FIT operator and Krylov solvers (arXiv 1705.08849).

The compute path is the CUDA library built from ``csrc/`` (C ABI in ``include/fit.h``);
``fit`` is its thin ctypes binding.
"""
from . import fit  # noqa: F401
from .fit import Grid, FitError  # noqa: F401
