"""Builds the CUDA library ``lib/libpi2rh.so`` in-tree for sm_103a (B300).

    python -m paper_1503_00330_b300.build            # build if sources changed
    python -m paper_1503_00330_b300.build --force    # rebuild

nvcc cross-compiles without a GPU.  ``-Xptxas -v`` output (registers, spills,
shared memory per kernel) is written to ``lib/ptxas.txt``.
"""
from __future__ import annotations

import glob
import os
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
LIBDIR = os.path.join(PKG, "lib")
LIB = os.path.join(LIBDIR, "libpi2rh.so")
INCLUDE = os.path.join(ROOT, "include")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xptxas", "-v",
              "--expt-relaxed-constexpr", "-cudart", "shared"]


def sources() -> list[str]:
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cuh"))
                  + glob.glob(os.path.join(CSRC, "*.h")) + [os.path.join(INCLUDE, "pi2rh.h")])


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(s) <= t for s in sources())


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and up_to_date():
        return LIB
    os.makedirs(LIBDIR, exist_ok=True)
    cus = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    tmp = LIB + f".{os.getpid()}.tmp"
    cmd = ["nvcc", *ARCH, *NVCC_FLAGS, "-I", INCLUDE, "-I", CSRC, "-shared", *cus, "-o", tmp]
    r = subprocess.run(cmd, capture_output=True, text=True)
    with open(os.path.join(LIBDIR, "ptxas.txt"), "w") as f:
        f.write(" ".join(cmd) + "\n" + r.stdout + r.stderr)
    if r.returncode != 0:
        sys.stderr.write(r.stdout + r.stderr)
        raise RuntimeError("nvcc failed building libpi2rh.so")
    if verbose:
        sys.stdout.write(r.stderr)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True)
