"""Build the CUDA library (libvmc.so) for sm_103a with nvcc, in-tree.

Each translation unit is compiled in parallel, then linked into one shared library with the
C ABI declared in include/vmc.h.
"""
from __future__ import annotations

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor
from pathlib import Path

PKG = Path(__file__).resolve().parent
ROOT = PKG.parent
SRC = PKG / "csrc"
BUILD = PKG / "_build"
LIB = BUILD / "libvmc.so"
SOURCES = ["api.cu", "lists.cu", "walkers.cu", "eloc.cu", "grad.cu", "noalloc.cu", "umma.cu", "probe.cu", "cps.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC,-fopenmp,-O2",
         "-I", str(ROOT / "include"), "-I", str(SRC)]


def _nvcc() -> str:
    cand = os.environ.get("NVCC") or "/usr/local/cuda/bin/nvcc"
    return cand if Path(cand).exists() else "nvcc"


def build(force: bool = False, verbose: bool = False, extra: list[str] | None = None) -> Path:
    BUILD.mkdir(exist_ok=True)
    deps = [SRC / f for f in SOURCES] + [SRC / "common.cuh", ROOT / "include" / "vmc.h"]
    newest = max(p.stat().st_mtime for p in deps)
    if not force and LIB.exists() and LIB.stat().st_mtime >= newest:
        return LIB
    nvcc = _nvcc()
    extra = extra or []

    def compile_one(name: str) -> Path:
        obj = BUILD / (name + ".o")
        cmd = [nvcc, *ARCH, *FLAGS, *extra, "-c", str(SRC / name), "-o", str(obj)]
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        subprocess.run(cmd, check=True)
        return obj

    with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = BUILD / f"libvmc.{os.getpid()}.so"
    cmd = [nvcc, *ARCH, "-shared", "-o", str(tmp), *map(str, objs), "-Xcompiler", "-fopenmp"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True,
          extra=["-Xptxas", "-v"] if "--ptxas" in sys.argv else None)
