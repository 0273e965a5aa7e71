"""Build the in-tree CUDA library libugks.so for sm_103a (GB300) with nvcc."""
from __future__ import annotations

import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
ROOT = os.path.dirname(HERE)
LIB = os.path.join(HERE, "libugks.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# host code without floating-point contraction: the velocity grid and the tables built on
# the host round the same way on x86 and aarch64 (GCC contracts a*b + c into an FMA on
# aarch64 in C++ by default, which moved a v = 0 node of an asymmetric grid off zero)
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-ffp-contract=off"]

SOURCES = ["ugks.cu"]


def _inputs():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files.append(os.path.join(ROOT, "include", "ugks.h"))
    return [f for f in files if f.endswith((".cu", ".cuh", ".h"))]


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile every translation unit in parallel, link libugks.so; returns its path."""
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= max(os.path.getmtime(f) for f in _inputs())):
        return LIB
    nvcc = os.environ.get("NVCC", "nvcc")
    objs, procs = [], []
    for src in SOURCES:
        obj = os.path.join(CSRC, os.path.splitext(src)[0] + f".{os.getpid()}.o")
        cmd = [nvcc, *ARCH, *FLAGS, "-c", os.path.join(CSRC, src), "-o", obj]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        procs.append(subprocess.Popen(cmd))
        objs.append(obj)
    rc = [p.wait() for p in procs]
    if any(rc):
        for o in objs:
            if os.path.exists(o):
                os.remove(o)
        raise RuntimeError(f"nvcc failed: {rc}")
    tmp = LIB + f".tmp{os.getpid()}"
    subprocess.check_call([nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"])
    for o in objs:
        os.remove(o)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
