"""Build libmotjvie.so in-tree for sm_103a (B300) with nvcc."""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libmotjvie.so")
# the cuFFT comparison product (timed beside the library's own product only)
CUFFT_LIB = os.path.join(HERE, "libmotcufft.so")
CUFFT_SRC = os.path.join(SRC, "cufft_compare.cu")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")

NVCC_FLAGS = [
    "-O3",
    "-std=c++17",
    "-gencode", "arch=compute_103a,code=sm_103a",
    "-lineinfo",
    "-Xcompiler", "-fPIC,-fopenmp",
    "-shared",
]


def sources():
    return [os.path.join(SRC, f) for f in sorted(os.listdir(SRC))
            if f.endswith((".cu", ".cuh")) and f != "cufft_compare.cu"] + [os.path.join(INCLUDE, "motjvie.h")]


def needs_build() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(s) > t for s in sources())


def build_cufft_compare(force: bool = False, verbose: bool = False) -> str:
    """libmotcufft.so: the cuFFT-based comparison product used by bench.py."""
    if not force and os.path.exists(CUFFT_LIB) and os.path.getmtime(CUFFT_LIB) >= os.path.getmtime(CUFFT_SRC):
        return CUFFT_LIB
    nvcc = os.environ.get("NVCC", "nvcc")
    cmd = [nvcc, *NVCC_FLAGS, "-o", CUFFT_LIB, CUFFT_SRC, "-lcufft"]
    if verbose:
        print(" ".join(cmd), file=sys.stderr)
    subprocess.check_call(cmd)
    return CUFFT_LIB


def build(force: bool = False, verbose: bool = False) -> str:
    build_cufft_compare(force, verbose)
    if not force and not needs_build():
        return LIB
    nvcc = os.environ.get("NVCC", "nvcc")
    cmd = [nvcc, *NVCC_FLAGS, "-o", LIB, os.path.join(SRC, "api.cu"), "-lgomp"]
    if verbose:
        print(" ".join(cmd), file=sys.stderr)
    subprocess.check_call(cmd)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True)
    print(LIB)
