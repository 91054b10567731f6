"""GB300-native batched Keplerian-constrained BLS transit search (arXiv:2302.01293).

The compute path is the CUDA library ``libqlpbls`` (C ABI in include/qlp_bls.h),
reached through the ctypes binding ``paper_2302_01293_gb300.qlpbls``. Importing
this package loads nothing; ``qlpbls.lib()`` builds (if needed) and loads the
library.
"""
__all__ = ["qlpbls", "build"]
