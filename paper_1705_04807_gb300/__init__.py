"""Exact modular matrix multiply on Morton-hybrid matrices for GB300 (sm_103a).

The compute path lives in ``libfm.so`` (CUDA kernels and host C++ behind the
C ABI of ``include/fm.h``); ``native`` is its ctypes binding. PyTorch is only
used by callers for device memory and streams.
"""

from .native import *  # noqa: F401,F403
from .native import EXPORTS, FmError, gf2_matrix, gf2_sub, lib, matrix, opts, sub  # noqa: F401

__version__ = "0.1.0"
