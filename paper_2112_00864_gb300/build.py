"""Build the bcfmm CUDA library for sm_103a (GB300) in-tree.

Each translation unit is compiled in parallel with nvcc, then linked into
``paper_2112_00864_gb300/_build/libbcfmm.so``.  No cmake; one -gencode.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libbcfmm.so")
SOURCES = ["api.cu", "kernels_fmm.cu", "kernels_near.cu", "kernels_aux.cu", "m2l_taylor.cu", "m2l_tc.cu", "mlp.cu", "setup.cpp"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def _flags(src: str):
    # host code: -ffp-contract=off keeps the FP64 setup (quadrature points,
    # octree decisions) independent of multiply-add fusion, the same on
    # x86_64 and aarch64
    common = ["-O3", "-std=c++17", "-Xcompiler", "-fPIC,-fopenmp,-O3,-ffp-contract=off", "-I", os.path.join(ROOT, "include")]
    if src.endswith(".cu"):
        # -ftz=true: no operand of the FP32 passes comes near the denormal
        # range, and it lets rsqrtf compile to the bare MUFU reciprocal root
        return ARCH + ["-lineinfo", "--expt-relaxed-constexpr", "-ftz=true"] + common
    return ["-x", "c++"] + common


def _compile(src: str, verbose: bool) -> str:
    obj = os.path.join(OUT, os.path.splitext(src)[0] + ".o")
    path = os.path.join(CSRC, src)
    deps = [path] + [os.path.join(CSRC, h) for h in os.listdir(CSRC) if h.endswith((".h", ".cuh"))]
    deps.append(os.path.join(ROOT, "include", "bcfmm.h"))
    if os.path.exists(obj) and os.path.getmtime(obj) >= max(os.path.getmtime(d) for d in deps):
        return obj
    cmd = [nvcc(), "-c", path, "-o", obj] + _flags(src)
    if verbose:
        print(" ".join(cmd), flush=True)
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
    if verbose and r.stderr.strip():
        print(r.stderr, file=sys.stderr)
    return obj


def build(verbose: bool = False) -> str:
    os.makedirs(OUT, exist_ok=True)
    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(lambda s: _compile(s, verbose), SOURCES))
    if not os.path.exists(LIB) or os.path.getmtime(LIB) < max(os.path.getmtime(o) for o in objs):
        tmp = LIB + f".{os.getpid()}.tmp"
        cmd = [nvcc(), "-shared", "-o", tmp] + objs + ARCH + ["-Xcompiler", "-fopenmp", "-lgomp"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(verbose=True))
