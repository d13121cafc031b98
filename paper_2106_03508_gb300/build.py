"""Build the AGF2 shared library (libagf2.so) in-tree with nvcc for sm_103a.

Each translation unit is compiled in parallel, then linked with cuSOLVER and
cuBLAS (used only for the O(N^3) FP64 steps).  Usage: ``python -m
paper_2106_03508_gb300.build`` or ``build()`` from Python.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor
from pathlib import Path

PKG = Path(__file__).resolve().parent
CSRC = PKG / "csrc"
INCLUDE = PKG.parent / "include"
OUT_DIR = PKG / "_build"
LIB = PKG / "libagf2.so"
SOURCES = ["capi.cu", "fp64.cu", "mixed.cu", "rotate.cu", "noalloc.cu", "eigen.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not Path(cand).exists():
        raise RuntimeError("nvcc not found; the AGF2 library needs the CUDA toolkit")
    return cand


def _flags(extra=()):
    return ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                   "-I", str(INCLUDE), "-I", str(CSRC), *extra]


def build(verbose: bool = False, force: bool = False, ptxas_verbose: bool = False) -> Path:
    nvcc = _nvcc()
    OUT_DIR.mkdir(exist_ok=True)
    deps = [CSRC / s for s in SOURCES] + list(CSRC.glob("*.h")) + list(CSRC.glob("*.cuh")) + \
        [INCLUDE / "agf2.h"]
    newest = max(p.stat().st_mtime for p in deps)
    if LIB.exists() and not force and LIB.stat().st_mtime > newest:
        return LIB
    extra = ["-Xptxas", "-v"] if ptxas_verbose else []

    def compile_one(src: str) -> Path:
        obj = OUT_DIR / (Path(src).stem + ".o")
        cmd = [nvcc, *_flags(extra), "-c", str(CSRC / src), "-o", str(obj)]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
        if verbose or ptxas_verbose:
            sys.stderr.write(r.stdout + r.stderr)
        return obj

    with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = LIB.with_suffix(".so.tmp")
    cmd = [nvcc, *ARCH, "-shared", "-o", str(tmp), *map(str, objs), "-lcusolver", "-lcublas", "-lpthread"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(verbose=True, force="--force" in sys.argv, ptxas_verbose="-v" in sys.argv))
