"""GB300 (sm_103a) MOT-JVIE marching library: FFT-accelerated, FIR-regularised
marching-on-in-time solver for the contrast-current-density volume integral
equation (arXiv 2407.03323).

The compute path is the CUDA library ``libmot.so`` (C ABI in include/mot.h); this
package holds its sources (``csrc/``), the build step (``build``) and the ctypes
binding (``mot``).
"""
from .mot import Context, MotError, load_library  # noqa: F401
