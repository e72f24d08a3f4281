"""In-tree build of libpeps.so (CUDA, sm_103a) with plain nvcc, no cmake.

The translation units compile in parallel; the shared library is written to
``paper_1611_09467_gb300/_lib/libpeps.so``.  Rebuilds only when a source is
newer than the library.  ``build(phase_timing=True)`` writes a separate
diagnostic library, ``_lib/phase/libpeps.so``, with the truncation's phase
counters compiled in (``phase_timing.py``); the library itself never has them.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_lib")
LIB = os.path.join(OUT, "libpeps.so")
PHASE_OUT = os.path.join(OUT, "phase")
PHASE_LIB = os.path.join(PHASE_OUT, "libpeps.so")
SOURCES = ["kernels.cu", "row.cu", "pair.cu", "mc.cu", "corr.cu", "su.cu", "peaks.cu", "api.cu", "serve.cu"]
INCLUDE = os.path.join(ROOT, "include")


def _headers():
    """Every header the sources can include: csrc/*.cuh, csrc/*.h and include/*.h
    (listed from the directories, so a new header cannot be left out)."""
    out = [os.path.join(CSRC, f) for f in sorted(os.listdir(CSRC)) if f.endswith((".cuh", ".h"))]
    if os.path.isdir(INCLUDE):
        out += [os.path.join(INCLUDE, f) for f in sorted(os.listdir(INCLUDE)) if f.endswith(".h")]
    return out

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2"]


def nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libpeps.so")


def _stale(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    deps = [os.path.join(CSRC, f) for f in SOURCES] + _headers() + [os.path.abspath(__file__)]
    return any(os.path.getmtime(d) > t for d in deps if os.path.exists(d))


def build(force: bool = False, verbose: bool = False, phase_timing: bool = False) -> str:
    out_dir, lib = (PHASE_OUT, PHASE_LIB) if phase_timing else (OUT, LIB)
    if not force and not _stale(lib):
        return lib
    os.makedirs(out_dir, exist_ok=True)
    cc = nvcc()
    objs = []
    extra = ["-DPEPS_PHASE_TIMING"] if phase_timing else []

    def compile_one(src):
        obj = os.path.join(out_dir, os.path.splitext(src)[0] + ".o")
        cmd = [cc, *ARCH, *FLAGS, *extra, "-c", os.path.join(CSRC, src), "-o", obj]
        if verbose:
            print(" ".join(cmd), flush=True)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        return obj

    with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = lib + ".tmp"
    cmd = [cc, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
