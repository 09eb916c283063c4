"""Compile the CUDA C-ABI library ``libgcb.so`` for sm_103a with nvcc.

The translation units are compiled in parallel and linked in-tree into
``paper_2007_14401_gb300/_lib/libgcb.so``; nothing is installed elsewhere.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUT_DIR = os.path.join(HERE, "_lib")
LIB = os.path.join(OUT_DIR, "libgcb.so")
OBJ_DIR = os.path.join(HERE, "_build")
# the measured arithmetic peaks of the benchmark (include/gcb_peak.h)
PEAK_LIB = os.path.join(OUT_DIR, "libgcb_peak.so")
PEAK_SRC = "peak_fma.cu"

SOURCES = ["gcb_api.cu", "sort_sr.cu", "gcb_noalloc.cu", "gcb_ks.cu", "adjoint_sr.cu",
           "push_sr_f64.cu", "push_sr_f32.cu", "push_dep_f64.cu", "push_dep_f32.cu",
           "push_mir_f64.cu", "push_mir_f32.cu"]
# The mixed-precision push and the adjoint unit use approximate FP32 division
# and square root (about 2 ulp) and flush FP32 denormals: the flags act on
# single precision only, so the FP64 kernels in the adjoint unit keep IEEE
# operations, as does the FP64 push.  The adjoint's FP32 replay of a step then
# uses the same arithmetic as the FP32 push it retraces.
EXTRA = {"push_sr_f32.cu": ["-use_fast_math"], "push_dep_f32.cu": ["-use_fast_math"],
         "push_mir_f32.cu": ["-use_fast_math"],
         "adjoint_sr.cu": ["-use_fast_math"]}
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVFLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-I" + INCLUDE, "-I" + CSRC]


def _nvcc() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found")
    return cand


def _deps_mtime() -> float:
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files.append(os.path.join(INCLUDE, "gcb.h"))
    return max(os.path.getmtime(f) for f in files)


def build_peak(force: bool = False) -> str:
    """Build libgcb_peak.so (the FMA-rate measurement) if needed; returns its path."""
    src = os.path.join(CSRC, PEAK_SRC)
    deps = max(os.path.getmtime(src), os.path.getmtime(os.path.join(INCLUDE, "gcb_peak.h")))
    if not force and os.path.exists(PEAK_LIB) and os.path.getmtime(PEAK_LIB) >= deps:
        return PEAK_LIB
    os.makedirs(OUT_DIR, exist_ok=True)
    tmp = PEAK_LIB + f".{os.getpid()}.tmp"
    cmd = [_nvcc(), *ARCH, *NVFLAGS, "-shared", src, "-o", tmp, "-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {PEAK_SRC}:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, PEAK_LIB)
    return PEAK_LIB


def build(force: bool = False, verbose: bool = False) -> str:
    """Build libgcb.so (and libgcb_peak.so) if missing or older than their
    sources; returns the path of libgcb.so."""
    build_peak(force)
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= _deps_mtime():
        return LIB
    os.makedirs(OUT_DIR, exist_ok=True)
    os.makedirs(OBJ_DIR, exist_ok=True)
    nvcc = _nvcc()

    def compile_one(src):
        obj = os.path.join(OBJ_DIR, src.replace(".cu", ".o"))
        cmd = [nvcc, *ARCH, *NVFLAGS, *EXTRA.get(src, []), "-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
        if verbose:
            print(r.stdout + r.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = LIB + f".{os.getpid()}.tmp"
    cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
