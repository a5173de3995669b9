"""Builds libtkf.so in-tree: every CUDA translation unit compiled for sm_103a in parallel
with nvcc, then linked into one shared library with a C ABI (include/tkf.h)."""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libtkf.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# Single-precision arithmetic in the kernels uses the fast forms (flush-to-zero, approximate
# division and square root, hardware sin/cos/log): measured against the FP64 reference CPU
# implementation, the FP32 errors of the whole path stay as they are with the exact forms
# (precision sweep test), and the build kernel runs about 20 % faster.  Double-precision
# arithmetic is not affected.
FAST_MATH = ["-use_fast_math"]
SOURCES = ["tkf_api.cu", "tkf_build_fp32.cu", "tkf_build_mixed.cu", "tkf_build_fp64.cu", "tkf_build2_fp32.cu",
           "tkf_build2_mixed.cu", "tkf_build2_fp64.cu", "tkf_build3_fp32.cu", "tkf_build3_mixed.cu",
           "tkf_build3_fp64.cu", "tkf_pipeline.cu", "tkf_server.cu", "tkf_probe.cu", "tkf_seeding.cu"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libtkf.so")


def _deps():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(INCLUDE, "tkf.h"), __file__]
    return max(os.path.getmtime(f) for f in files if os.path.exists(f))


def _compile(src: str, extra: list[str]) -> str:
    obj = os.path.join(BUILD, os.path.splitext(src)[0] + ".o")
    cmd = [nvcc(), *ARCH, "-O3", "-lineinfo", "-std=c++17", *FAST_MATH, "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I",
           CSRC, "-c", os.path.join(CSRC, src), "-o", obj, *extra]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (src, " ".join(cmd), r.stderr[-6000:]))
    return obj


def build(force: bool = False, verbose: bool = False, extra: list[str] | None = None) -> str:
    """Compile (if stale) and return the path of libtkf.so."""
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= _deps():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    extra = list(extra or [])
    srcs = [s for s in SOURCES if os.path.exists(os.path.join(CSRC, s))]
    with cf.ThreadPoolExecutor(max_workers=len(srcs)) as ex:
        objs = list(ex.map(lambda s: _compile(s, extra), srcs))
    tmp = LIB + ".%d.tmp" % os.getpid()
    cmd = [nvcc(), *ARCH, "-shared", "-o", tmp, *objs, "-lpthread"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s\n%s" % (" ".join(cmd), r.stderr[-4000:]))
    os.replace(tmp, LIB)
    if verbose:
        print("built", LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True, extra=["-Xptxas", "-v"] if "--ptxas" in sys.argv else None)
