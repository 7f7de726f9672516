"""GB300-native Parareal for periodic advection-diffusion (arXiv:1409.8563).

The compute path lives in a C-ABI shared library (``include/parareal.h``)
built from ``csrc/``; ``paper_1409_8563_gb300.native`` is its thin ctypes
binding.  Importing this package loads nothing: the library is opened on
first use and a missing library is an error, never a fallback.
"""
__all__ = ["native", "inputs", "configs"]
