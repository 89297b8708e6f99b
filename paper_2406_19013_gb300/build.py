"""Builds libcorr.so in-tree with nvcc for sm_103a (no cmake, no torch build).

The translation units compile in parallel; the CUDA runtime is linked
statically and the driver's tensor-map encoder is looked up at run time, so
the library loads on a machine without a GPU driver (it then fails at
corr_create with CORR_ECUDA).
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libcorr.so")
# The debug variant (CORR_DEBUG: address checks in the kernels, guard bands
# around the integration buffers) builds into its own folder and library.
BUILD_DEBUG = os.path.join(HERE, "_build_debug")
LIB_DEBUG = os.path.join(HERE, "libcorr_debug.so")
SOURCES = ["xengine.cu", "xengine_tm.cu", "dump.cu", "corr.cu", "corr_static.cu", "xe_sched.cu", "batch.cu", "corner_turn.cu", "server.cu", "fengine.cu", "mma_peak.cu"]
HEADERS = ["ptx.cuh", "xe_internal.h", "xe_sched.h", "xe_unpack.cuh", "trace.h"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-Wall", "-I", INCLUDE]


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libcorr.so")


def _inputs():
    root = os.path.dirname(HERE)
    deps = [os.path.join(CSRC, f) for f in SOURCES + HEADERS]
    deps.append(os.path.join(root, "include", "corr.h"))
    deps.append(os.path.abspath(__file__))
    return deps


def up_to_date(debug: bool = False) -> bool:
    lib = LIB_DEBUG if debug else LIB
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(d) <= t for d in _inputs())


def build(force: bool = False, verbose: bool = False, debug: bool = False) -> str:
    """Builds libcorr.so (or, with debug=True, libcorr_debug.so) if any input
    is newer than it; returns the library's path."""
    lib, bdir = (LIB_DEBUG, BUILD_DEBUG) if debug else (LIB, BUILD)
    if not force and up_to_date(debug):
        return lib
    nvcc = _nvcc()
    os.makedirs(bdir, exist_ok=True)
    flags = FLAGS + (["-DCORR_DEBUG"] if debug else [])
    procs = []
    for src in SOURCES:
        obj = os.path.join(bdir, src.replace(".cu", ".o"))
        cmd = [nvcc, *ARCH, *flags, "-c", os.path.join(CSRC, src), "-o", obj]
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        procs.append((cmd, obj, subprocess.Popen(cmd, stdout=subprocess.PIPE,
                                                 stderr=subprocess.STDOUT)))
    objs = []
    failed = []
    for cmd, obj, pr in procs:
        out, _ = pr.communicate()
        if pr.returncode != 0:
            failed.append((cmd, out.decode(errors="replace")))
        objs.append(obj)
    if failed:
        msg = "\n".join(" ".join(c) + "\n" + o for c, o in failed)
        raise RuntimeError("nvcc failed:\n" + msg)
    tmp = lib + f".tmp{os.getpid()}"
    subprocess.run([nvcc, *ARCH, "-shared", "-cudart", "static", *objs, "-o", tmp], check=True)
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv, debug="--debug" in sys.argv))
