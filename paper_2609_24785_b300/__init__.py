"""B300-native ghost-point IBM / ADE impedance / 2D linearized Euler solver.

The compute path lives in ``liblee.so`` (CUDA kernels for sm_103a and a C++
host set-up behind the C ABI of ``include/lee.h``); ``lee`` is its ctypes
binding.  Importing the package does not load the library; ``lee.load()``
does, and raises if it is missing (there is no CPU fallback).
"""
__all__ = ["lee", "workloads", "build"]
