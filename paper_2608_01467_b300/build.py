"""Builds libfeynsparse.so in-tree with nvcc for sm_103a.

    python -m paper_2608_01467_b300.build [--force]
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libfeynsparse.so")
SOURCES = [os.path.join(CSRC, f) for f in ("fs_host.cpp", "fs_jit.cpp", "fs_kernels.cu", "fs_mlp.cu", "fs_noalloc.cu")]
DEPS = SOURCES + [os.path.join(CSRC, "fs_internal.h"), os.path.join(ROOT, "include", "feynsparse.h")]
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def needs_build(lib=LIB, deps=DEPS) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and not needs_build():
        return LIB
    cmd = [NVCC, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
           "-Xcompiler", "-fvisibility=hidden", "-shared", "-cudart", "shared",
           "-I", os.path.join(ROOT, "include"), "-o", LIB + ".tmp", *SOURCES,
           "-L/usr/local/cuda/lib64", "-lnvrtc", "-Xlinker", "-rpath=/usr/local/cuda/lib64"]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
        print(" ".join(cmd))
    subprocess.check_call(cmd)
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose="-v" in sys.argv)
    print(LIB)
