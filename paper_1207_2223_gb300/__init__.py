"""GB300 (sm_103a) library for two-flavour Wilson-fermion Hybrid Monte Carlo.

The compute path is the CUDA library built from ``csrc/`` (C interface in
``include/lq.h``); ``lq`` is a thin ctypes binding with the same function
names that only marshals arguments.  There is no CPU fallback: importing
the binding fails loudly when the library has not been built.
"""
from . import lq  # noqa: F401
from .lq import *  # noqa: F401,F403
