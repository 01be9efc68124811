"""Builds libres2tac.so (the CUDA library behind include/res2tac.h) in-tree with nvcc.

Only sm_103a code is generated (GB300). Each translation unit compiles in parallel; the link
step uses nvcc's default static CUDA runtime so the library loads without a matching libcudart
on the library path.
"""
from __future__ import annotations

import concurrent.futures
import glob
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OBJDIR = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libres2tac.so")
# The debug build with range checks in the aggregation and WTA kernels (RES2TAC_CHECK_BOUNDS)
CHECK_OBJDIR = os.path.join(HERE, "_build_check")
CHECK_LIB = os.path.join(HERE, "libres2tac_check.so")
UNITS = ("abi.cu", "kernels_plain.cu", "kernels_batch.cu", "noalloc.cu", "agg_rows_narrow.cu",
         "agg_rows_wide.cu", "agg_shear_narrow.cu", "agg_shear_wide.cu", "agg_shear_batch_narrow.cu",
         "agg_shear_batch_wide.cu", "ncc.cu", "rectify.cu", "cost_mma.cu")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I" + INCLUDE]


def nvcc() -> str:
    exe = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(exe):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libres2tac.so")
    return exe


def _sources():
    return (glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cuh")) +
            glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(INCLUDE, "*.h")))


def is_stale(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    return any(os.path.getmtime(s) > t for s in _sources())


def build(force: bool = False, verbose: bool = False, check: bool = False) -> str:
    """Compile and link the library if a source changed (or force). Returns the .so path.
    check=True builds the debug library with range checks (libres2tac_check.so) instead."""
    lib, objdir = (CHECK_LIB, CHECK_OBJDIR) if check else (LIB, OBJDIR)
    extra = ["-DRES2TAC_CHECK_BOUNDS"] if check else []
    if not force and not is_stale(lib):
        return lib
    os.makedirs(objdir, exist_ok=True)
    exe = nvcc()

    def compile_unit(unit):
        obj = os.path.join(objdir, unit.replace(".cu", ".o"))
        cmd = [exe, *ARCH, *FLAGS, *extra, "-c", os.path.join(CSRC, unit), "-o", obj]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {unit}:\n{r.stdout}\n{r.stderr}")
        return obj, r.stderr

    with concurrent.futures.ThreadPoolExecutor(len(UNITS)) as ex:
        results = list(ex.map(compile_unit, UNITS))
    if verbose:
        for _, log in results:
            print(log)
    tmp = lib + f".tmp{os.getpid()}"
    cmd = [exe, *ARCH, "-shared", "-o", tmp, *[o for o, _ in results]]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
