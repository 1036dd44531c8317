"""Builds liblee.so (CUDA kernels for sm_103a + the C++ host set-up and C ABI)
in-tree with nvcc."""
from __future__ import annotations

import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "liblee.so")
SOURCES = ["lee_kernels.cu", "lee_setup.cpp", "lee_api.cpp", "lee_noalloc.cu", "lee_measure.cu"]
HEADERS = ["lee_internal.h", os.path.join("..", "..", "include", "lee.h")]

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build liblee")


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, f) for f in SOURCES + HEADERS]
    return any(os.path.getmtime(p) > t for p in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and not _stale():
        return LIB
    srcs = [os.path.join(CSRC, f) for f in SOURCES]
    tmp = LIB + ".tmp"
    cmd = [nvcc(), "-O3", "-std=c++17", "-shared", "-lineinfo", *ARCH,
           "-Xcompiler", "-fPIC,-fopenmp,-ffp-contract=off,-Wall",
           "-Xptxas", "-v" if verbose else "-O3",
           "-o", tmp, *srcs, "-lgomp"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    import sys
    build(force=True, verbose="-v" in sys.argv)
    print(LIB)
