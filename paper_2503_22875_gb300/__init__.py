"""GB300-native FP64 / complex128 GEMM emulated with INT8-range slices on the tensor cores
(the Ozaki scheme with a tunable split number, arXiv 2503.22875).

The compute path is the CUDA library ``libozg.so`` (C ABI in ``include/ozg.h``); ``ozg`` is
its thin ctypes binding and ``workloads`` holds the seeded synthetic input generators.
Importing this package does not load the library; ``ozg.load()`` does, and fails loudly if
it has not been built.
"""
__all__ = ["ozg", "workloads", "build"]
