"""Builds the CUDA library ``libgks.so`` in-tree for sm_103a (GB300).

nvcc compiles ``csrc/gks.cu`` (kernels and the C ABI of ``include/gks.h``) into a shared
library next to this file.  The build is skipped when the library is newer than every
source.  No CPU fallback is built.
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
LIB = os.path.join(HERE, "libgks.so")
SOURCES = [os.path.join(HERE, "csrc", n) for n in ("gks.cu", "gks_batch.cu", "gks_tools.cu")]
DEPS = SOURCES + [os.path.join(HERE, "csrc", "gks_device.cuh"), os.path.join(HERE, "csrc", "gks_grid.cuh"),
                  os.path.join(ROOT, "include", "gks.h")]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.isabs(cand) and os.path.exists(cand) or not os.path.isabs(cand)):
            return cand
    return "nvcc"


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and os.path.exists(LIB):
        if os.path.getmtime(LIB) >= max(os.path.getmtime(p) for p in DEPS):
            return LIB
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [nvcc(), "-O3", "-std=c++17", *ARCH, "-lineinfo", "-Xcompiler", "-fPIC", "-shared", "--threads", "3",
           "-diag-suppress", "20011,20014",
           "-I", os.path.join(ROOT, "include"), "-o", tmp, *SOURCES]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
        print(" ".join(cmd), file=sys.stderr)
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose="-v" in sys.argv)
    print(LIB)
