"""GB300-native factored Levenberg-Marquardt LNCC registration.

The compute path is liblmreg.so (hand-written sm_103a CUDA kernels behind the
C ABI of include/lmreg.h); ``lmreg`` is its thin ctypes binding.
"""
from . import lmreg  # noqa: F401
from .lmreg import *  # noqa: F401,F403
