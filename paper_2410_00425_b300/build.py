"""Build libmsim.so (the C ABI of include/ms.h) for sm_103a, in place, and
its bounds-checked twin libmsim_debug.so (-DMS_DEBUG_BOUNDS: the stages'
index invariants checked after the narrowphase and the colouring, a
violation reported as MS_ENV_BOUNDS instead of an out-of-range access).

Every translation unit compiles to its own object in parallel (the batched
kernel once per lane-group size G, from ms_fused.cu with -DMS_FUSED_G=G);
the objects link into the shared library.

    python -m paper_2410_00425_b300.build [--force] [--debug] [--all]
"""
from __future__ import annotations

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OBJ = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libmsim.so")
LIB_DEBUG = os.path.join(HERE, "libmsim_debug.so")
SOURCES = ["ms_api.cu", "ms_kernels.cu", "ms_noalloc.cu", "ms_server.cu", "ms_render.cu", "ms_peak.cu"]
FUSED = "ms_fused.cu"
FUSED_G = (1, 2, 4, 8, 16, 32)
HEADERS = ["ms_math.cuh", "ms_narrow.cuh", "ms_stages.cuh", "ms_internal.h"]
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# -fmad=false: every fused multiply-add is written out in the source, so the
# rounding does not depend on how a stage is inlined into a kernel.
# -prec-div=false: the compiler's approximate float division (at most 2 ulp
# from the rounded quotient) instead of IEEE-rounded division; every kernel
# of the library is built the same way, so the plain, batched, server and
# no-allocation paths keep agreeing bit for bit.
FLAGS = ARCH + ["-lineinfo", "-O3", "-std=c++17", "-fmad=false", "-prec-div=false", "-Xcompiler", "-fPIC",
                "--expt-relaxed-constexpr"]


def _newest_input() -> float:
    paths = [os.path.join(CSRC, f) for f in SOURCES + [FUSED] + HEADERS]
    paths.append(os.path.join(os.path.dirname(HERE), "include", "ms.h"))
    paths.append(os.path.join(os.path.dirname(HERE), "include", "ms_server.h"))
    paths.append(os.path.abspath(__file__))
    return max(os.path.getmtime(p) for p in paths)


def _jobs(debug: bool):
    """(object path, nvcc command) of every translation unit of one library."""
    tag = "dbg" if debug else "rel"
    extra = ["-DMS_DEBUG_BOUNDS"] if debug else []
    jobs = []
    for f in SOURCES:
        o = os.path.join(OBJ, f"{tag}_{f[:-3]}.o")
        jobs.append((o, [NVCC] + FLAGS + extra + ["-c", os.path.join(CSRC, f), "-o", o]))
    for G in FUSED_G:
        o = os.path.join(OBJ, f"{tag}_ms_fused_g{G}.o")
        jobs.append((o, [NVCC] + FLAGS + extra + [f"-DMS_FUSED_G={G}", "-c", os.path.join(CSRC, FUSED), "-o", o]))
    return jobs


def _stale(lib: str, force: bool) -> bool:
    return force or not os.path.exists(lib) or os.path.getmtime(lib) < _newest_input()


def build_libs(debug_flags=(False,), force: bool = False, verbose: bool = False) -> list:
    """Build the requested libraries (False: release, True: debug) with all
    their objects compiled in one parallel pool; returns their paths."""
    todo = [d for d in debug_flags if _stale(LIB_DEBUG if d else LIB, force)]
    os.makedirs(OBJ, exist_ok=True)
    jobs = {d: _jobs(d) for d in todo}
    every = [j for d in todo for j in jobs[d]]

    def run(job):
        if verbose:
            print(" ".join(job[1]), flush=True)
        r = subprocess.run(job[1], capture_output=True, text=True)
        return job, r

    failed = []
    with ThreadPoolExecutor(max_workers=max(1, os.cpu_count() or 1)) as ex:
        for job, r in ex.map(run, every):
            if r.returncode != 0:
                failed.append((job, r))
            elif verbose and r.stderr.strip():
                print(r.stderr, file=sys.stderr)
    if failed:
        job, r = failed[0]
        raise RuntimeError(f"nvcc failed ({' '.join(job[1])}):\n{r.stdout}\n{r.stderr}")
    for d in todo:
        lib = LIB_DEBUG if d else LIB
        tmp = lib + ".tmp"
        cmd = [NVCC] + ARCH + ["-shared", "-o", tmp] + [o for o, _ in jobs[d]]
        if verbose:
            print(" ".join(cmd), flush=True)
        subprocess.check_call(cmd)
        os.replace(tmp, lib)
    return [LIB_DEBUG if d else LIB for d in debug_flags]


def build(force: bool = False, verbose: bool = False, debug: bool = False) -> str:
    """Build the library (debug: the bounds-checked one) unless it is newer
    than every source; returns its path."""
    return build_libs((debug,), force=force, verbose=verbose)[0]


if __name__ == "__main__":
    flags = (False, True) if "--all" in sys.argv else ("--debug" in sys.argv,)
    print(build_libs(flags, force="--force" in sys.argv, verbose=True))
