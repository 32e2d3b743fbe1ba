"""libmotjvie: B300-native MOT-JVIE solver with a matrix-free FFT product for Z0.

The compute path lives in the CUDA library ``libmotjvie.so`` (built from
``csrc/`` for sm_103a); this package is a thin ctypes binding with the same
names as the C ABI in ``include/motjvie.h``.  There is no CPU fallback: if the
library is missing or no CUDA device is present, the calls raise.
"""
from .binding import *  # noqa: F401,F403
from .binding import __all__  # noqa: F401
