"""GB300-native interpolated stencil multigrid (ISM) pressure solver.

The numerical path lives in the CUDA library ``libism.so`` (``csrc/``,
C ABI in ``include/ism.h``); ``ism`` is its thin ctypes binding.
"""
from . import ism  # noqa: F401  (binding only; the library loads on first use)

__all__ = ["ism"]
