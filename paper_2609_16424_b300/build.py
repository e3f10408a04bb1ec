"""Build the in-tree shared library ``liblh.so`` from ``csrc/*.cu`` for sm_103a (B300).

Usage: ``python paper_2609_16424_b300/build.py [--force] [-v]`` (run by path, so that a
stale library is never loaded while building).  Objects go to
``_build/`` at the repository root; the library is written next to this file so that
it travels with the source tree.
"""
import concurrent.futures as cf
import glob
import os
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
OUT = os.path.join(PKG, "liblh.so")
OBJ = os.path.join(ROOT, "_build")
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-Wall",
         "-diag-suppress", "177"]


def _deps():
    return sorted(glob.glob(os.path.join(CSRC, "*")) + [os.path.join(ROOT, "include", "lh.h")])


def _compile(src, verbose):
    obj = os.path.join(OBJ, os.path.basename(src).replace(".cu", ".o"))
    newest = max(os.path.getmtime(p) for p in _deps())
    if os.path.exists(obj) and os.path.getmtime(obj) >= newest:
        return obj
    extra = []
    if os.path.basename(src) == "lh_flops.cu":
        # the operation counter instantiates __host__ __device__ code with a host-only scalar
        extra = ["-diag-suppress", "20011,20014"]
    cmd = [NVCC] + ARCH + FLAGS + extra + ["-c", src, "-o", obj]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
        print(" ".join(cmd), flush=True)
    subprocess.run(cmd, check=True)
    return obj


def build(force=False, verbose=False):
    """Compile every CUDA source and link ``liblh.so``; return its path."""
    os.makedirs(OBJ, exist_ok=True)
    srcs = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    if force:
        for o in glob.glob(os.path.join(OBJ, "*.o")):
            os.remove(o)
    with cf.ThreadPoolExecutor(max_workers=min(8, len(srcs))) as ex:
        objs = list(ex.map(lambda s: _compile(s, verbose), srcs))
    newest = max(os.path.getmtime(o) for o in objs)
    if force or not os.path.exists(OUT) or os.path.getmtime(OUT) < newest:
        cmd = [NVCC] + ARCH + ["-shared", "-cudart", "shared", "-o", OUT] + objs + [
            "-Xlinker", "-rpath=/usr/local/cuda/lib64"]
        if verbose:
            print(" ".join(cmd), flush=True)
        subprocess.run(cmd, check=True)
    return OUT


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
