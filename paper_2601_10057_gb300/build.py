"""Build the in-tree CUDA library ``libccmsav.so`` for sm_103a with nvcc.

The translation units (the C ABI, the FP32-bulk and the FP64 instantiations
of the step, the allocation-free mass and the standalone spectral solver) are
compiled in parallel and linked into one shared object
next to this file.  ``python -m paper_2601_10057_gb300.build`` runs it.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libccmsav.so")
LIB_BOUNDS = os.path.join(HERE, "libccmsav_bounds.so")   # index-checked build (-DCCMSAV_BOUNDS), for tests
SOURCES = ["ccmsav_api.cu", "sim_f32.cu", "sim_f64.cu", "ccmsav_noalloc.cu", "spectral_solve.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr"]


def nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _newest(paths):
    return max(os.path.getmtime(p) for p in paths)


def build(force: bool = False, verbose: bool = False, bounds: bool = False) -> str:
    """Compile (if needed) and return the path of libccmsav.so; with
    bounds=True the index-checked libccmsav_bounds.so (-DCCMSAV_BOUNDS)."""
    lib = LIB_BOUNDS if bounds else LIB
    bdir = os.path.join(BUILD, "bounds") if bounds else BUILD
    extra = ["-DCCMSAV_BOUNDS"] if bounds else []
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    deps.append(os.path.join(HERE, "..", "include", "ccmsav.h"))
    if not force and os.path.exists(lib) and os.path.getmtime(lib) >= _newest(deps):
        return lib
    os.makedirs(bdir, exist_ok=True)
    cc = nvcc()

    def compile_one(src):
        obj = os.path.join(bdir, src.replace(".cu", ".o"))
        cmd = [cc, *ARCH, *FLAGS, *extra, "-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
        if verbose:
            sys.stdout.write(r.stdout + r.stderr)
        return obj

    with cf.ThreadPoolExecutor(len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = lib + ".tmp"
    cmd = [cc, *ARCH, "-shared", "-cudart", "shared", *objs, "-o", tmp]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv, bounds="--bounds" in sys.argv))
