"""Build libmsim.so (the C ABI of include/ms.h) for sm_103a, in place, and
its bounds-checked twin libmsim_debug.so (-DMS_DEBUG_BOUNDS: the stages'
index invariants checked after the narrowphase and the colouring, a
violation reported as MS_ENV_BOUNDS instead of an out-of-range access).

    python -m paper_2410_00425_b300.build [--force] [--debug]
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libmsim.so")
LIB_DEBUG = os.path.join(HERE, "libmsim_debug.so")
SOURCES = ["ms_api.cu", "ms_kernels.cu", "ms_noalloc.cu", "ms_server.cu", "ms_render.cu"]
HEADERS = ["ms_math.cuh", "ms_narrow.cuh", "ms_stages.cuh", "ms_internal.h"]
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
# -fmad=false: every fused multiply-add is written out in the source, so the
# rounding does not depend on how a stage is inlined into a kernel
FLAGS = ["-gencode", "arch=compute_103a,code=sm_103a", "-lineinfo", "-O3", "-std=c++17", "-fmad=false",
         "-Xcompiler", "-fPIC", "-shared", "--expt-relaxed-constexpr"]


def _newest_input() -> float:
    paths = [os.path.join(CSRC, f) for f in SOURCES + HEADERS]
    paths.append(os.path.join(os.path.dirname(HERE), "include", "ms.h"))
    paths.append(os.path.join(os.path.dirname(HERE), "include", "ms_server.h"))
    paths.append(os.path.abspath(__file__))
    return max(os.path.getmtime(p) for p in paths)


def build(force: bool = False, verbose: bool = False, debug: bool = False) -> str:
    """Build the library (debug: the bounds-checked one) unless it is newer
    than every source; returns its path."""
    lib = LIB_DEBUG if debug else LIB
    if not force and os.path.exists(lib) and os.path.getmtime(lib) >= _newest_input():
        return lib
    tmp = lib + ".tmp"
    cmd = [NVCC] + FLAGS + (["-DMS_DEBUG_BOUNDS"] if debug else []) + ["-o", tmp] + \
        [os.path.join(CSRC, f) for f in SOURCES]
    if verbose:
        print(" ".join(cmd))
    subprocess.check_call(cmd)
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, debug="--debug" in sys.argv))
