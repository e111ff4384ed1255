"""GB300-native hot path of auto-weighted robust tensor-ring decomposition (AWRTRD /
SAWRTRD with FGMC and RStS; He & Atia, UAI 2023).

The compute lives in libtrd.so (CUDA kernels for sm_103a behind the C ABI of
include/trd.h); `binding` marshals arguments to it, `synth` draws seeded workloads.
The library is loaded lazily so that the workload generator imports without a GPU.
"""
from .binding import TRD, TrdError, draw_indices, load, ring_cut  # noqa: F401

__all__ = ["TRD", "TrdError", "draw_indices", "load", "ring_cut"]
