"""B300-native SGSPM hot path: C-ABI library `libsgspm.so` (hand-written sm_103a CUDA)
plus a thin ctypes binding.

Importing the package is cheap; the library is loaded by `paper_2606_28113_b300.sgspm`
on first use and the binding raises if it is missing (there is no CPU fallback).
"""
__all__ = ["inputs", "sgspm"]
