"""Build the tFFR CUDA library (csrc/*.cu -> _tffr.so) for sm_103a, in-tree.

Three translation units (the C ABI with the point/spread kernels, the FFT
line kernels, the persistent batch kernels) compiled in parallel, one
-gencode, static CUDA runtime.
"""

from __future__ import annotations

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "_tffr.so")
SOURCES = [os.path.join(CSRC, "tffr.cu"), os.path.join(CSRC, "line_kernels.cu"), os.path.join(CSRC, "batch.cu")]
DEPS = SOURCES + [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))] + [
    os.path.join(ROOT, "include", "tffr.h"), os.path.abspath(__file__)]

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
CFLAGS = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC"]


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    return "nvcc"


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and os.path.exists(LIB):
        t = os.path.getmtime(LIB)
        if all(os.path.getmtime(d) <= t for d in DEPS if os.path.exists(d)):
            return LIB
    tag = "%d" % os.getpid()
    objs = [os.path.join(CSRC, os.path.basename(s)[:-3] + ".%s.o" % tag) for s in SOURCES]
    extra = ["-Xptxas", "-v"] if verbose else []

    def compile_one(args):
        src, obj = args
        subprocess.run([nvcc()] + CFLAGS + extra + ["-c", src, "-o", obj], check=True)

    try:
        with ThreadPoolExecutor(len(SOURCES)) as ex:
            list(ex.map(compile_one, zip(SOURCES, objs)))
        tmp = LIB + ".tmp" + tag
        subprocess.run([nvcc()] + ARCH + ["-shared", "-cudart", "static"] + objs + ["-o", tmp], check=True)
        os.replace(tmp, LIB)
    finally:
        for o in objs:
            if os.path.exists(o):
                os.remove(o)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
