"""Builds the CUDA library libebpoisson.so in-tree for sm_103a (GB300).

Six translation units compiled in parallel: geometry.cu (setup work, no FMA
contraction so the cut-cell geometry is bit-reproducible), solver.cu
(multigrid kernels, driver, C ABI), server.cu (the serving loop, host code),
amr.cu (the composite solve over nested refined boxes), tga.cu (TGA
diffusion steps) and tagging.cu (refinement tags, no FMA contraction).  The CUDA runtime is linked statically.
"""
from __future__ import annotations

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libebpoisson.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
UNITS = {"geometry.cu": ["--fmad=false"], "solver.cu": [], "server.cu": [], "amr.cu": [], "tga.cu": [], "tagging.cu": ["--fmad=false"]}


def _nvcc():
    cuda = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    p = os.path.join(cuda, "bin", "nvcc")
    return p if os.path.exists(p) else "nvcc"


def _sources():
    return [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [
        os.path.join(os.path.dirname(HERE), "include", "ebpoisson.h")]


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(s) <= t for s in _sources())


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and up_to_date():
        return LIB
    os.makedirs(OUT_DIR, exist_ok=True)
    nvcc = _nvcc()
    common = ARCH + ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
                     "-I", os.path.join(os.path.dirname(HERE), "include")]

    def compile_one(item):
        src, extra = item
        obj = os.path.join(OUT_DIR, src.replace(".cu", ".o"))
        cmd = [nvcc] + common + extra + ["-c", os.path.join(CSRC, src), "-o", obj]
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        subprocess.check_call(cmd)
        return obj

    with ThreadPoolExecutor(max_workers=len(UNITS)) as ex:
        objs = list(ex.map(compile_one, UNITS.items()))
    tmp = LIB + f".tmp{os.getpid()}"
    subprocess.check_call([nvcc] + ARCH + ["-shared", "-o", tmp] + objs)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
