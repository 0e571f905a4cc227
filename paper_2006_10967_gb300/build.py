"""Compile libfrpcpf.so in-tree for sm_103a (nvcc for CUDA, g++ for host C++).

Translation units compile in parallel; the library is rebuilt only when a
source or header is newer than it.
"""
import concurrent.futures as cf
import glob
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libfrpcpf.so")
ROOT = os.path.dirname(HERE)

NVCC = os.environ.get("NVCC", "nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVFLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC"] + ARCH
CXXFLAGS = ["-O2", "-std=c++17", "-fPIC"]

CU = ["api.cu", "k_quad.cu", "k_hex.cu", "k_tri.cu", "k_group.cu", "noalloc.cu", "adjoint.cu"]
# The residual/update kernels' float arithmetic (the mixed path) uses the
# approximate reciprocal, division and square root (2 ulp) and flushes
# denormals; FP64 arithmetic is unaffected by these flags.
FAST_FLOAT = ["-ftz=true", "-prec-div=false", "-prec-sqrt=false"]
FAST_FLOAT_TU = {"k_quad.cu", "k_hex.cu", "k_tri.cu", "k_group.cu"}
CPP = ["mesh.cpp", "refel.cpp"]


def _sources():
    return [os.path.join(CSRC, f) for f in CU + CPP]


def _deps():
    return _sources() + glob.glob(os.path.join(CSRC, "*.h*")) + glob.glob(os.path.join(CSRC, "*.cuh")) + \
        [os.path.join(ROOT, "include", "fr_pcpf.h"), __file__]


def stale():
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(d) > t for d in _deps() if os.path.exists(d))


def _compile(src):
    obj = os.path.join(BUILD, os.path.basename(src) + ".o")
    if src.endswith(".cu"):
        extra = FAST_FLOAT if os.path.basename(src) in FAST_FLOAT_TU else []
        cmd = [NVCC] + NVFLAGS + extra + ["-c", src, "-o", obj]
    else:
        cmd = ["g++"] + CXXFLAGS + ["-c", src, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"compile failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    return obj


def build(force=False, verbose=False):
    """Build libfrpcpf.so if stale (or force); return its path."""
    if not force and not stale():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    with cf.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 4)) as ex:
        objs = list(ex.map(_compile, _sources()))
    tmp = LIB + ".tmp"
    cmd = [NVCC] + ARCH + ["-shared", "-o", tmp] + objs
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    if verbose:
        print("built", LIB, file=sys.stderr)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True)
