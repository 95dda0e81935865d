"""Builds libwsim.so (the CUDA library behind include/wsim.h) for sm_103a.

nvcc cross-compiles without a GPU.  The library is built in-tree, next to
this file, so that it travels with the source tree.
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
SO = os.path.join(HERE, "libwsim.so")
SOURCES = ["wsim_kernels.cu", "wsim_rollout.cu", "wsim_bptt.cu", "wsim_observe.cu", "wsim_route.cu", "wsim_api.cu", "wsim_static.cu"]
HEADERS = ["wsim_device.cuh", "wsim_internal.h", "wsim_phases.cuh"]
NVCC_FLAGS = ["-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-lineinfo", "-std=c++17",
              "-Xcompiler", "-fPIC", "-shared"]


def _inputs():
    files = [os.path.join(CSRC, f) for f in SOURCES + HEADERS]
    files.append(os.path.join(ROOT, "include", "wsim.h"))
    return files


def stale() -> bool:
    if not os.path.exists(SO):
        return True
    t = os.path.getmtime(SO)
    return any(os.path.getmtime(f) > t for f in _inputs())


def build(force: bool = False, verbose: bool = False) -> str:
    if force or stale():
        cmd = ["nvcc", *NVCC_FLAGS, *(["-Xptxas", "-v"] if verbose else []), "-o", SO,
               *[os.path.join(CSRC, f) for f in SOURCES]]
        subprocess.check_call(cmd)
    return SO


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose="-v" in sys.argv)
    print(SO)
