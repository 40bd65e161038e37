"""Build the CUDA library libecris.so in-tree for sm_103a (GB300).

Each translation unit is compiled by nvcc in parallel, then linked into one
shared library beside this file.  No GPU is needed to build.
"""
from __future__ import annotations

import concurrent.futures
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libecris.so")
SOURCES = ["api.cu", "step_kernel.cu", "coulomb.cu", "coulomb_noalloc.cu", "sort.cu", "server.cu", "probe.cu",
           "ne_update.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--cudart", "shared"]
# The step kernels for one run and for a batch inline the same per-particle
# code; without contraction of separate multiplies and adds into FMAs (an
# optimiser's choice that may differ between the two kernels) both round
# every operation the same way, so a run gives identical results alone and in
# a batch.  Explicit fmaf() calls in that code still compile to FMAs.
# The device update of n_e builds the cell records in FP64 as the host does,
# operation by operation, so it is compiled without contraction too.  So is
# the collision kernel: its shared-memory and global-memory paths inline the
# same collision arithmetic, and a cell goes to one or the other depending on
# how the cells fall into ranges; without contraction both round the same.
FILE_FLAGS = {"step_kernel.cu": ["-fmad=false"], "ne_update.cu": ["-fmad=false"], "coulomb.cu": ["-fmad=false"]}


def _nvcc():
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.isabs(cand) and os.path.exists(cand) or not os.path.isabs(cand)):
            return cand
    return "nvcc"


def _stale(target, deps):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(BUILD, exist_ok=True)
    headers = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    headers.append(os.path.join(HERE, "..", "include", "ecris.h"))
    headers.append(os.path.abspath(__file__))   # flag changes rebuild everything
    nvcc = _nvcc()
    jobs = []
    objs = []
    for src in SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(BUILD, src.replace(".cu", ".o"))
        objs.append(o)
        if force or _stale(o, [s] + headers):
            cmd = [nvcc, *ARCH, *FLAGS, *FILE_FLAGS.get(src, []), "-c", s, "-o", o]
            if verbose:
                cmd.insert(1, "-Xptxas=-v")
            jobs.append(cmd)

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
        return r.stdout + r.stderr

    with concurrent.futures.ThreadPoolExecutor(max_workers=max(1, len(jobs))) as ex:
        outs = list(ex.map(run, jobs))
    if verbose:
        for o in outs:
            print(o)
    if force or jobs or _stale(LIB, objs):
        run([nvcc, *ARCH, "-shared", "--cudart", "shared", *objs, "-o", LIB])
    return LIB


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
