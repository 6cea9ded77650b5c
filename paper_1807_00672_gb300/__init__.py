"""GB300-native HLLC finite-volume shallow-water step (Zaoui, arXiv 1807.00672).

The compute path is the CUDA library ``libswe.so`` (kernels for sm_103a behind
a C ABI, declared in ``include/swe.h``); ``swe`` is its ctypes binding and
``inputs`` the seeded synthetic workloads. Importing the package loads nothing:
``swe`` loads the library on first use and raises if it is missing.
"""
__all__ = ["inputs", "swe"]
