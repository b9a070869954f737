"""Build libecg.so in-tree with nvcc for sm_103a (GB300).

Three translation units (the single-system solver, the batched solver and
the warm-start network),
compiled in parallel with one -gencode each and linked into one library;
the library links the CUDA runtime statically so that it loads next to any
PyTorch build.
"""
from __future__ import annotations

import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(HERE, "libecg.so")
SOURCES = [os.path.join(CSRC, "ecg.cu"), os.path.join(CSRC, "batch.cu"), os.path.join(CSRC, "nn.cu")]
DEPS = SOURCES + [
    os.path.join(CSRC, "ecg_kernels.cuh"),
    os.path.join(CSRC, "ecg_batch.cuh"),
    os.path.join(INCLUDE, "ecg.h"),
    os.path.join(INCLUDE, "ecg_nn.h"),
]
OBJDIR = os.path.join(HERE, "_build")
FLAGS = ["-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libecg.so")


def needs_build() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(d) > t for d in DEPS)


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and not needs_build():
        return LIB
    os.makedirs(OBJDIR, exist_ok=True)
    tag = f"{os.getpid()}"
    objs, procs = [], []
    for src in SOURCES:
        obj = os.path.join(OBJDIR, os.path.splitext(os.path.basename(src))[0] + f".{tag}.o")
        cmd = [nvcc(), *FLAGS, "-I" + INCLUDE, "-c", "-o", obj, src]
        if verbose:
            print(" ".join(cmd))
        procs.append(subprocess.Popen(cmd))
        objs.append(obj)
    rcs = [p.wait() for p in procs]
    try:
        if any(rcs):
            raise subprocess.CalledProcessError(max(rcs), "nvcc -c")
        tmp = LIB + f".tmp{tag}"
        cmd = [nvcc(), "-gencode", "arch=compute_103a,code=sm_103a", "-shared", "-o", tmp, *objs]
        if verbose:
            print(" ".join(cmd))
        subprocess.check_call(cmd)
        os.replace(tmp, LIB)
    finally:
        for o in objs:
            if os.path.exists(o):
                os.remove(o)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
