"""Compile the CUDA library ``libhashpoint.so`` in-tree for sm_103a, and its
bounds-check build ``libhashpoint_checks.so`` (-DHP_CHECKS=1: every checked
gather / scatter index is tested before the access, a failure recorded as
HP_ERR_BOUNDS and the access skipped).

Run as ``python -m paper_2404_14044_b300.build`` (or through
``__graft_entry__.build()``).  nvcc cross-compiles without a GPU.
"""
from __future__ import annotations

import glob
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
LIB = os.path.join(HERE, "libhashpoint.so")
LIB_CHECKS = os.path.join(HERE, "libhashpoint_checks.so")
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def sources():
    return sorted(glob.glob(os.path.join(HERE, "csrc", "*.cu")))


def headers():
    return sorted(glob.glob(os.path.join(HERE, "csrc", "*.cuh"))) + [os.path.join(ROOT, "include", "hashpoint.h")]


def up_to_date(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(f) <= t for f in sources() + headers() + [__file__])


def build(force: bool = False, verbose: bool = False, checks: bool = False) -> str:
    lib = LIB_CHECKS if checks else LIB
    if not force and up_to_date(lib):
        return lib
    cmd = [NVCC, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-shared",
           "-I", os.path.join(ROOT, "include"), "-cudart", "shared",
           "-Xlinker", "-rpath,/usr/local/cuda/lib64", "-o", lib + ".tmp", *sources()]
    if checks:
        cmd.insert(1, "-DHP_CHECKS=1")
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    subprocess.run(cmd, check=True)
    os.replace(lib + ".tmp", lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
    print(build(force="--force" in sys.argv, checks=True))
