"""Builds libcusadi.so in-tree: host C++ with g++, device code for sm_103a with nvcc.

Translation units are compiled in parallel and the library is linked against
the static CUDA runtime and NVRTC; the driver API is reached through the
runtime's entry-point query, so the library also loads on machines without a
GPU driver (code generation and compilation then still work).
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OBJ = os.path.join(ROOT, "_build", "obj")
LIB = os.path.join(HERE, "libcusadi.so")
CUDA = os.environ.get("CUDA_HOME", "/usr/local/cuda")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]

HOST_SRC = ["ir.cpp", "passes.cpp", "codegen.cpp", "coop.cpp", "interp.cpp", "runtime.cpp", "batch.cpp"]
DEVICE_SRC = ["kernels.cu", "noalloc.cu"]


def _sources():
    return [os.path.join(CSRC, f) for f in HOST_SRC + DEVICE_SRC] + [
        os.path.join(CSRC, "internal.h"), os.path.join(INCLUDE, "cusadi.h")]


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(s) > t for s in _sources())


def _compile(src: str) -> str:
    obj = os.path.join(OBJ, os.path.basename(src) + ".o")
    if src.endswith(".cu"):
        cmd = [os.path.join(CUDA, "bin", "nvcc"), *ARCH, "-lineinfo", "-O3", "-std=c++17",
               "-Xcompiler", "-fPIC", "-I", INCLUDE, "-c", src, "-o", obj]
    else:
        cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-Wall", "-I", INCLUDE,
               "-I", os.path.join(CUDA, "include"), "-c", src, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"compile failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    return obj


def build(force: bool = False) -> str:
    """Compile (if sources changed) and return the path of libcusadi.so."""
    if not force and not _stale():
        return LIB
    os.makedirs(OBJ, exist_ok=True)
    srcs = [os.path.join(CSRC, f) for f in DEVICE_SRC + HOST_SRC]
    with ThreadPoolExecutor(max_workers=len(srcs)) as ex:
        objs = list(ex.map(_compile, srcs))
    lib64 = os.path.join(CUDA, "lib64")
    tmp = LIB + ".tmp"
    cmd = ["g++", "-shared", "-o", tmp, *objs, "-L", lib64, "-lcudart_static", "-lnvrtc", "-lnvJitLink",
           "-lpthread", "-ldl", "-lrt", f"-Wl,-rpath,{lib64}"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
