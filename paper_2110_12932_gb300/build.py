"""Compile the CUDA library ``libtl.so`` in-tree for sm_103a (GB300).

The library has two translation units (csrc/tl_api.cu, the two-level path,
and csrc/tl_noalloc.cu, the allocation-free single step), compiled in
parallel; it links the CUDA runtime statically, so the only run-time
dependency is the NVIDIA driver's libcuda.
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
    """Build libtl.so unless it is newer than every source; returns its path.
    The translation units compile in parallel (nvcc -c), then link."""
    if not force and up_to_date():
        return LIB
    compile_flags = [f for f in NVCC_FLAGS if f != "-shared"]
    inc = ["-I", os.path.join(ROOT, "include")]
    objs, procs = [], []
    for src in SOURCES:
        obj = os.path.join(HERE, os.path.basename(src).replace(".cu", ".o"))
        cmd = [nvcc(), *compile_flags, *inc, "-c", "-o", obj, src]
        if verbose:
            print(" ".join(cmd))
        procs.append(subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True))
        objs.append(obj)
    failed = []
    for proc in procs:
        out, _ = proc.communicate()
        if proc.returncode != 0:
            failed.append(out)
    if failed:
        raise RuntimeError("nvcc failed:\n" + "\n".join(failed))
    tmp = LIB + ".tmp"
    cmd = [nvcc(), "-gencode", "arch=compute_103a,code=sm_103a", "-shared", "-Xcompiler", "-fPIC", "-o", tmp, *objs]
    if verbose:
        print(" ".join(cmd))
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError("nvcc link failed:\n" + res.stdout + res.stderr)
    os.replace(tmp, LIB)
    for obj in objs:
        os.remove(obj)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
