"""cgflow: GB300-native FP64 right-hand side of the compressible Euler equations
with C-GBR, LAD and hybrid LAD-GBR shock capturing (arXiv 2511.18042).

The compute path is the CUDA library ``_build/libcgflow.so`` (C ABI in
``include/cgflow.h``); ``api`` is its thin Python binding.
"""
from . import inputs  # noqa: F401
