"""Compile libfrpcpf.so in-tree for sm_103a (nvcc for CUDA, g++ for host C++).

Translation units compile in parallel; the library is rebuilt only when a
source or header is newer than it.  build(checked=True) compiles the same
sources with FR_BOUNDS_CHECK defined into libfrpcpf_checked.so: every
partner index read from the connectivity is checked on the device before it
is used (an index out of range gives FR_EBOUNDS, and no access leaves the
arrays).  The package loads the checked library when the environment sets
FRP_BOUNDS_CHECK=1.
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
LIB_CHECKED = os.path.join(HERE, "libfrpcpf_checked.so")
BUILD_CHECKED = os.path.join(HERE, "_build_checked")
ROOT = os.path.dirname(HERE)

NVCC = os.environ.get("NVCC", "nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVFLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC"] + ARCH
CXXFLAGS = ["-O2", "-std=c++17", "-fPIC"]

CU = ["api.cu", "k_quad.cu", "k_hex.cu", "k_tri.cu", "k_group.cu", "noalloc.cu", "adjoint.cu", "probe_dense.cu"]
# The residual/update kernels' float arithmetic (the mixed path) uses the
# approximate reciprocal, division and square root (2 ulp) and flushes
# denormals; FP64 arithmetic is unaffected by these flags.
FAST_FLOAT = ["-ftz=true", "-prec-div=false", "-prec-sqrt=false"]
FAST_FLOAT_TU = {"k_quad.cu", "k_hex.cu", "k_tri.cu", "k_group.cu", "probe_dense.cu"}
CPP = ["mesh.cpp", "refel.cpp"]


def _sources():
    return [os.path.join(CSRC, f) for f in CU + CPP]


def _deps():
    return _sources() + glob.glob(os.path.join(CSRC, "*.h*")) + glob.glob(os.path.join(CSRC, "*.cuh")) + \
        [os.path.join(ROOT, "include", "fr_pcpf.h"), __file__]


def _target(checked):
    return (LIB_CHECKED, BUILD_CHECKED) if checked else (LIB, BUILD)


def stale(checked=False):
    lib = _target(checked)[0]
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    return any(os.path.getmtime(d) > t for d in _deps() if os.path.exists(d))


def _compile(src, checked=False):
    obj = os.path.join(_target(checked)[1], os.path.basename(src) + ".o")
    if src.endswith(".cu"):
        extra = FAST_FLOAT if os.path.basename(src) in FAST_FLOAT_TU else []
        if checked:
            extra = extra + ["-DFR_BOUNDS_CHECK"]
        cmd = [NVCC] + NVFLAGS + extra + ["-c", src, "-o", obj]
    else:
        cmd = ["g++"] + CXXFLAGS + ["-c", src, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"compile failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    return obj


def build_all(force=False, verbose=False, checked=(False, True)):
    """Build the libraries named by checked (plain and/or bounds-checked),
    their translation units compiled in one parallel pool; return the paths."""
    todo = [c for c in checked if force or stale(c)]
    if todo:
        jobs = [(src, c) for c in todo for src in _sources()]
        for c in todo:
            os.makedirs(_target(c)[1], exist_ok=True)
        with cf.ThreadPoolExecutor(max_workers=min(16, os.cpu_count() or 4)) as ex:
            objs = list(ex.map(lambda j: _compile(*j), jobs))
        for c in todo:
            lib = _target(c)[0]
            mine = [o for o, (_, cj) in zip(objs, jobs) if cj == c]
            tmp = lib + ".tmp"
            cmd = [NVCC] + ARCH + ["-shared", "-o", tmp] + mine
            r = subprocess.run(cmd, capture_output=True, text=True)
            if r.returncode != 0:
                raise RuntimeError(f"link failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
            os.replace(tmp, lib)
            if verbose:
                print("built", lib, file=sys.stderr)
    return [_target(c)[0] for c in checked]


def build(force=False, verbose=False, checked=False):
    """Build libfrpcpf.so (or, with checked, libfrpcpf_checked.so) if stale
    (or force); return its path."""
    return build_all(force, verbose, (checked,))[0]


if __name__ == "__main__":
    build_all(force="--force" in sys.argv, verbose=True,
              checked=(False, True) if "--checked" in sys.argv else (False,))
