"""Build step of the CUDA library: nvcc, sm_103a only, in-tree.

``python -m paper_1110_1379_gb300.build`` (or ``build()``) compiles every
translation unit under ``csrc/`` in parallel and links
``paper_1110_1379_gb300/_build/libfrmg.so``.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libfrmg.so")
SOURCES = ["frmg_solver.cu", "frmg_cic.cu", "frmg_noalloc.cu", "frmg_poisson.cu",
           "frmg_masked.cu", "frmg_symmetron.cu"]
HEADERS = ["frmg_kernels.cuh", "frmg_df.cuh", "frmg_dfmath.cuh", "frmg_internal.h"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc():
    exe = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(exe):
        raise RuntimeError("nvcc not found")
    return exe


def _stale():
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, s) for s in SOURCES + HEADERS]
    deps.append(os.path.join(ROOT, "include", "frmg.h"))
    deps.append(os.path.abspath(__file__))
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, extra=()) -> str:
    if not force and not _stale():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    common = [nvcc(), "-O3", "-std=c++17", "-lineinfo", *ARCH, "-Xcompiler", "-fPIC",
              "-I", os.path.join(ROOT, "include"), "-I", CSRC, *extra]
    procs = []
    objs = []
    try:
        for s in SOURCES:
            obj = os.path.join(BUILD, s.replace(".cu", f".{os.getpid()}.o"))
            objs.append(obj)
            cmd = common + ["-c", os.path.join(CSRC, s), "-o", obj]
            if verbose:
                print(" ".join(cmd))
            procs.append(subprocess.Popen(cmd))
        failed = [p.wait() != 0 for p in procs]
        if any(failed):
            raise RuntimeError("nvcc failed")
        tmp = LIB + f".tmp{os.getpid()}"
        link = [nvcc(), *ARCH, "-shared", "-o", tmp, *objs]
        subprocess.run(link, check=True)
        os.replace(tmp, LIB)
    finally:
        for p in procs:
            if p.poll() is None:
                p.wait()
        for o in objs:
            if os.path.exists(o):
                os.remove(o)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True)
    print(LIB)
