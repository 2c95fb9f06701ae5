"""GB300 session discrimination + millisecond histogramming (arXiv 2106.12863).

The compute path is the CUDA library ``_lib/libsinet.so`` (C ABI in
include/sinet.h); this package is its Python binding.
"""
from .sinet import *  # noqa: F401,F403
from .sinet import load  # noqa: F401
