"""Compile the CUDA library ``libtl.so`` in-tree for sm_103a (GB300).

The library has two translation units (csrc/tl_api.cu, the two-level path,
and csrc/tl_noalloc.cu, the allocation-free single step); it links the CUDA
runtime statically, so the only run-time dependency is the NVIDIA driver's
libcuda.
"""
from __future__ import annotations

import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
LIB = os.path.join(HERE, "libtl.so")
SOURCES = [os.path.join(HERE, "csrc", "tl_api.cu"), os.path.join(HERE, "csrc", "tl_noalloc.cu")]
DEPS = SOURCES + [os.path.join(HERE, "csrc", f) for f in ("tl_device.cuh", "tl_solve.cuh")] + [
    os.path.join(ROOT, "include", "tl.h")]

NVCC_FLAGS = [
    "-gencode", "arch=compute_103a,code=sm_103a",
    "-O3", "-lineinfo", "-std=c++17", "--extended-lambda",
    "-Xcompiler", "-fPIC", "-shared",
]


def nvcc():
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libtl.so")


def up_to_date():
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(d) <= t for d in DEPS if os.path.exists(d))


def build(force=False, verbose=False):
    """Build libtl.so unless it is newer than every source; returns its path."""
    if not force and up_to_date():
        return LIB
    tmp = LIB + ".tmp"
    cmd = [nvcc(), *NVCC_FLAGS, "-I", os.path.join(ROOT, "include"), "-o", tmp, *SOURCES]
    if verbose:
        print(" ".join(cmd))
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError("nvcc failed:\n" + res.stdout + res.stderr)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
