"""GB300-native (sm_103a) DF-EA-ADC(3) sigma vectors and Davidson solver.

The compute lives in libeaadc.so (hand-written CUDA behind the C ABI of
include/eaadc.h); ``_lib`` is its ctypes binding.  Importing this package does
not load the library; the first call does, and fails if it is missing.
"""
from ._lib import *  # noqa: F401,F403
from ._lib import lib, EaadcError, EXPORTED, LIB_PATH  # noqa: F401
