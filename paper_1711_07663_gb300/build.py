"""Build libdirectcut.so in-tree for sm_103a (GB300) with nvcc.

    python -m paper_1711_07663_gb300.build          # or build() from Python

The library is written to paper_1711_07663_gb300/_build/libdirectcut.so.
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
LIB = os.path.join(BUILD, "libdirectcut.so")
SOURCES = ["dc_api.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libdirectcut")


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(ROOT, "include", "directcut.h")]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(BUILD, exist_ok=True)
    if not force and not _stale():
        return LIB
    tmp = LIB + f".{os.getpid()}.tmp"
    cmd = [_nvcc(), *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-shared",
           "-o", tmp] + [os.path.join(CSRC, s) for s in SOURCES]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
        print(" ".join(cmd), file=sys.stderr)
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


PEAKS_SRC = os.path.join(ROOT, "bench_peaks.cu")
PEAKS_LIB = os.path.join(ROOT, "_build", "libbenchpeaks.so")


def build_peaks(force: bool = False) -> str:
    """The benchmark's FP32/FP64 FMA peak microbenchmark (bench_peaks.cu at the
    repository root) into _build/libbenchpeaks.so; not part of the library."""
    os.makedirs(os.path.dirname(PEAKS_LIB), exist_ok=True)
    if not force and os.path.exists(PEAKS_LIB) and os.path.getmtime(PEAKS_LIB) >= os.path.getmtime(PEAKS_SRC):
        return PEAKS_LIB
    tmp = PEAKS_LIB + f".{os.getpid()}.tmp"
    subprocess.run([_nvcc(), *ARCH, "-O3", "-lineinfo", "-Xcompiler", "-fPIC", "-shared", "-o", tmp, PEAKS_SRC],
                   check=True)
    os.replace(tmp, PEAKS_LIB)
    return PEAKS_LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
