"""Build ``libtled.so`` in-tree with nvcc for sm_103a (B300).

``python -m paper_2009_10400_b300.build`` or ``build()`` from Python.  The
library is a plain C-ABI shared object (include/tled.h); the Python binding
loads it with ctypes.
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libtled.so")
SOURCES = ["tled_host.cpp", "tled_capi.cpp", "tled_kernels.cu", "tled_noalloc.cu", "mlp_capi.cpp", "mlp_kernels.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    deps.append(os.path.join(HERE, "..", "include", "tled.h"))
    deps.append(os.path.join(HERE, "..", "include", "tled_mlp.h"))
    return any(os.path.getmtime(d) > t for d in deps if os.path.exists(d))


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and not _stale():
        return LIB
    cmd = [NVCC, "-O3", "-std=c++17", "-shared", "-Xcompiler", "-fPIC,-O3", *ARCH, "-lineinfo",
           "--expt-relaxed-constexpr", "-o", LIB + ".tmp", *[os.path.join(CSRC, s) for s in SOURCES]]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    subprocess.check_call(cmd)
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
