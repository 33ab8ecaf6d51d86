"""Build ``libtled.so`` in-tree with nvcc for sm_103a (B300).

``python -m paper_2009_10400_b300.build`` or ``build()`` from Python.  The
library is a plain C-ABI shared object (include/tled.h, include/tled_mlp.h);
the Python binding loads it with ctypes.  Each source compiles to an object
under ``_build/`` (in parallel, only when it or a header changed), then one
link step makes the library.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OBJ = os.path.join(ROOT, "_build")
LIB = os.path.join(HERE, "libtled.so")
SOURCES = ["tled_host.cpp", "tled_capi.cpp", "tled_kernels.cu", "tled_noalloc.cu", "mlp_capi.cpp", "mlp_kernels.cu",
           "sur_capi.cpp"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
FLAGS = ["-O3", "-std=c++17", "-Xcompiler", "-fPIC,-O3", *ARCH, "-lineinfo", "--expt-relaxed-constexpr"]


def _headers():
    hs = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".h")]
    return hs + [os.path.join(ROOT, "include", f) for f in os.listdir(os.path.join(ROOT, "include"))]


def _mtime(p):
    return os.path.getmtime(p) if os.path.exists(p) else -1.0


def _obj(src):
    return os.path.join(OBJ, src + ".o")


def _compile(src, verbose):
    cmd = [NVCC, *FLAGS, "-c", "-o", _obj(src) + ".tmp", os.path.join(CSRC, src)]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    subprocess.check_call(cmd)
    os.replace(_obj(src) + ".tmp", _obj(src))


def build(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(OBJ, exist_ok=True)
    newest_header = max(_mtime(h) for h in _headers())
    stale = [s for s in SOURCES
             if force or verbose or _mtime(_obj(s)) < max(_mtime(os.path.join(CSRC, s)), newest_header)]
    if stale:
        with cf.ThreadPoolExecutor(max_workers=len(stale)) as ex:
            for f in [ex.submit(_compile, s, verbose) for s in stale]:
                f.result()
    if stale or _mtime(LIB) < max(_mtime(_obj(s)) for s in SOURCES):
        subprocess.check_call([NVCC, "-shared", *ARCH, "-o", LIB + ".tmp", *[_obj(s) for s in SOURCES]])
        os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
