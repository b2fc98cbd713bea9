"""GB300-native periodic tricubic B-spline orbital evaluation (arXiv:1611.02665).

The compute path is the CUDA library built from ``csrc/`` behind the C ABI
of ``include/bspline_gb300.h``; ``capi`` is its thin ctypes binding.
Importing this package loads nothing; the library is loaded on first use.
"""
from . import capi  # noqa: F401
from .capi import (BF16, F16, F32, V, VGH, VGL, Table, BsplineError)  # noqa: F401
