"""GB300-native lid-driven cavity: SSPRK(5,4) vorticity / stream-function step.

The compute path is the CUDA library built from ``csrc/`` (C ABI in
``include/lc.h``); ``lc`` is its ctypes binding and ``workloads`` holds the
benchmark configurations and seeded input generators.
"""
from . import lc, workloads  # noqa: F401
from .lc import Cavity  # noqa: F401
