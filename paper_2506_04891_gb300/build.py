"""Builds the in-tree CUDA library libqlayer.so for sm_103a.

Each translation unit is compiled by its own nvcc process (in parallel) and
then linked; no cmake.  Run ``python -m paper_2506_04891_gb300.build``.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "libqlayer.so")
BUILD_DIR = os.path.join(HERE, "_build")
SOURCES = ["qc_tile_bwd.cu", "qc_tile_fwd.cu", "qc_tile_tma_bwd.cu", "qc_tile_tma_fwd.cu", "qc_tile_tc.cu", "qc_kernels.cu",
           "qc_api.cu", "qc_noalloc.cu", "qc_peaks.cu"]
# the kernel files compile once per precision (QC_INST_R = 4 float, 8 double),
# so the two halves build in parallel
SPLIT = {"qc_tile_bwd.cu", "qc_tile_fwd.cu", "qc_kernels.cu"}


def _units():
    for src in SOURCES:
        if src in SPLIT:
            yield src, "_r4", ["-DQC_INST_R=4"]
            yield src, "_r8", ["-DQC_INST_R=8"]
        else:
            yield src, "", []
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc_path() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found (set NVCC or put CUDA's bin on PATH)")


def _compile(nvcc: str, unit, extra) -> str:
    src, tag, defs = unit
    obj = os.path.join(BUILD_DIR, os.path.splitext(src)[0] + tag + ".o")
    cmd = [nvcc, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-fvisibility=hidden",
           "--expt-relaxed-constexpr", *defs, "-c", os.path.join(CSRC, src), "-o", obj, *extra]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
    if r.stderr.strip():
        sys.stderr.write(r.stderr)
    return obj


def build(verbose: bool = False, extra=()) -> str:
    nvcc = nvcc_path()
    os.makedirs(BUILD_DIR, exist_ok=True)
    units = list(_units())
    with cf.ThreadPoolExecutor(max_workers=len(units)) as ex:
        objs = list(ex.map(lambda u: _compile(nvcc, u, list(extra)), units))
    tmp = OUT + ".tmp"
    cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, OUT)
    if verbose:
        print(f"built {OUT}")
    return OUT


if __name__ == "__main__":
    extra = sys.argv[1:]
    build(verbose=True, extra=extra)
