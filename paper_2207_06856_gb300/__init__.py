"""GB300-native low-precision Gaussian-process solves (matrix-free kernel MVM
inside enhanced-stability preconditioned CG).

The compute path lives in the CUDA library ``libgpk.so`` (C ABI declared in
``include/gpk.h``); :mod:`.gpk` is the thin ctypes binding over it.  Importing
this package does not load the library; the first call into :mod:`.gpk` does,
and raises if the library has not been built.
"""

__all__ = ["gpk", "workloads"]
