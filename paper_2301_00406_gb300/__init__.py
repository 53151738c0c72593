"""GB300 (sm_103a) curvature-regularised confocal NLOS reconstruction.

The compute lives in libnlos.so (CUDA kernels behind the C ABI of
include/nlos.h); ``nlos`` is its ctypes binding.
"""

from . import nlos  # noqa: F401
