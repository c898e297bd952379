"""Build the StaRMAP CUDA library (libstarmap.so) in-tree for sm_103a.

Each translation unit is compiled in parallel (nvcc for .cu, g++ for .cpp)
into ``_build/`` and linked into ``lib/libstarmap.so`` next to this file.
The CUDA runtime is linked statically, so the library loads on machines
without a GPU driver (the symbol-export tests run there).
"""
from __future__ import annotations

import concurrent.futures
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIBDIR = os.path.join(HERE, "lib")
LIB = os.path.join(LIBDIR, "libstarmap.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O2",
                     "--expt-relaxed-constexpr", "-I", CSRC]
CXX_FLAGS = ["-O2", "-fPIC", "-std=c++17", "-I", CSRC]

SOURCES = ["host_math.cpp", "kernels_gather.cu", "tiled.cu", "capi.cu", "noalloc.cu", "mlp.cu", "mlp_tc.cu", "mlp_capi.cu"]
HEADERS = ["host_math.h", "internal.h", "tiled.h", "tiled_kernel.cuh", "fused_kernel.cuh", "mlp.h", "closure_features.cuh",
           "pdl.h"]


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _deps_mtime() -> float:
    files = [os.path.join(CSRC, f) for f in HEADERS]
    files.append(os.path.join(os.path.dirname(HERE), "include", "starmap.h"))
    return max(os.path.getmtime(f) for f in files if os.path.exists(f))


def _compile(src: str, extra: list, verbose: bool) -> str:
    path = os.path.join(CSRC, src)
    obj = os.path.join(BUILD, src + ".o")
    if (os.path.exists(obj) and os.path.getmtime(obj) >= os.path.getmtime(path)
            and os.path.getmtime(obj) >= _deps_mtime()):
        return obj
    if src.endswith(".cu"):
        cmd = [_nvcc(), "-c", path, "-o", obj] + NVCC_FLAGS + extra
    else:
        cmd = [os.environ.get("CXX", "g++"), "-c", path, "-o", obj] + CXX_FLAGS + [
            "-I", "/usr/local/cuda/include"]
    if verbose:
        print(" ".join(cmd), flush=True)
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"compiling {src} failed:\n{res.stdout}\n{res.stderr}")
    if verbose and res.stderr.strip():
        print(res.stderr, file=sys.stderr)
    return obj


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False) -> str:
    """Compile every translation unit and link libstarmap.so; returns its path."""
    os.makedirs(BUILD, exist_ok=True)
    os.makedirs(LIBDIR, exist_ok=True)
    if force:
        for f in os.listdir(BUILD):
            if f.endswith(".o"):
                os.remove(os.path.join(BUILD, f))
    extra = ["-Xptxas", "-v"] if ptxas_info else []
    with concurrent.futures.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(lambda s: _compile(s, extra, verbose or ptxas_info), SOURCES))
    newest = max(os.path.getmtime(o) for o in objs)
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < newest:
        cmd = [_nvcc(), "-shared", "-o", LIB] + objs + ARCH + ["-lrt", "-ldl", "-lpthread"]
        if verbose:
            print(" ".join(cmd), flush=True)
        res = subprocess.run(cmd, capture_output=True, text=True)
        if res.returncode != 0:
            raise RuntimeError(f"linking libstarmap.so failed:\n{res.stdout}\n{res.stderr}")
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, ptxas_info="--ptxas" in sys.argv))
