"""GB300-native kernel quantile regression (PALM-KQR hot path).

The compute path is the CUDA library ``_build/libkqr.so`` (sm_103a) behind the
C ABI declared in ``include/kqr.h``; ``paper_2510_07929_gb300.kqr`` is its thin
ctypes binding.  Importing the package itself loads nothing, so the data
generators in ``workloads`` stay usable on machines without a GPU.
"""
__all__ = ["workloads", "kqr"]
