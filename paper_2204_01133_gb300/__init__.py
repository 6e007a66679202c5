"""GB300-native asynchrony-tolerant (AT) finite-difference RK-stage solver.

The compute path is the CUDA library ``libat_gb300.so`` (sm_103a) behind the
C ABI declared in ``include/at.h``; :mod:`paper_2204_01133_gb300.api` is the
thin ctypes binding.  Importing this package does not load the library; the
first call through the binding does, and raises if it is missing.
"""
__all__ = ["api", "workloads"]
