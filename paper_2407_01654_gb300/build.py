"""Builds the CUDA library libehd.so in-tree for sm_103a (GB300).

Each translation unit is compiled by nvcc in parallel, then linked into one shared
library with the CUDA runtime linked statically.  Usage: python -m
paper_2407_01654_gb300.build [--verbose] [--ptxas-info] [--checked]

--checked builds libehd_checked.so instead (-DEHD_CHECKED): the kernels test the indices
they form from lattice coordinates, count any out of range (ehd_diag_index_errors) and
clamp it, for debugging; it is slower and not what the benchmark runs.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libehd.so")
LIB_CHECKED = os.path.join(HERE, "libehd_checked.so")
SOURCES = ["kernels.cu", "poisson.cu", "poisson_resident.cu", "noalloc.cu", "batch.cu", "api.cu",
           "diag.cu", "slabs.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
         "--expt-relaxed-constexpr", "-I", os.path.join(ROOT, "include")]
# kernels.cu holds each pass twice, as a one-simulation kernel and as a batched kernel that
# reads its parameters from a table; with multiply-add contraction left to the compiler the
# two can round differently.  Without contraction both compute the same bits.  (The
# potential loop kernels write their roundings explicitly instead.)
FILE_FLAGS = {"kernels.cu": ["-fmad=false"]}


def nvcc():
    exe = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(exe):
        raise RuntimeError("nvcc not found")
    return exe


def _run(cmd, verbose):
    if verbose:
        print(" ".join(cmd), flush=True)
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"command failed ({r.returncode}): {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    return r.stdout + r.stderr


def build(verbose=False, ptxas_info=False, force=False, checked=False):
    """Compiles the library if a source is newer than it (or force).  Returns its path.
    checked: the index-checking debug build (libehd_checked.so)."""
    lib = LIB_CHECKED if checked else LIB
    bdir = BUILD_DIR + ("_checked" if checked else "")
    os.makedirs(bdir, exist_ok=True)
    srcs = [os.path.join(CSRC, s) for s in SOURCES]
    deps = srcs + [os.path.join(CSRC, "ehd_internal.cuh"), os.path.join(CSRC, "sim_internal.h"),
                   os.path.join(ROOT, "include", "ehd.h"), os.path.abspath(__file__)]
    if (not force and os.path.exists(lib)
            and all(os.path.getmtime(lib) >= os.path.getmtime(d) for d in deps)):
        return lib
    extra = ["-Xptxas", "-v"] if ptxas_info else []
    if checked:
        extra = extra + ["-DEHD_CHECKED"]
    objs = []
    cmds = []
    for s in srcs:
        o = os.path.join(bdir, os.path.basename(s).replace(".cu", ".o"))
        objs.append(o)
        cmds.append([nvcc(), *ARCH, *FLAGS, *FILE_FLAGS.get(os.path.basename(s), []), *extra,
                     "-c", s, "-o", o])
    with cf.ThreadPoolExecutor(max_workers=len(cmds)) as ex:
        outs = list(ex.map(lambda c: _run(c, verbose), cmds))
    if ptxas_info:
        for o in outs:
            print(o)
    tmp = lib + ".tmp"
    # -ldl: the header-only NVTX ranges look their tool up with dlopen
    _run([nvcc(), *ARCH, "-shared", "-cudart", "static", "-o", tmp, *objs, "-ldl"], verbose)
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(verbose="--verbose" in sys.argv, ptxas_info="--ptxas-info" in sys.argv,
                force=True, checked="--checked" in sys.argv))
