"""Build the CUDA library in-tree: ``_build/libbsq.so`` for sm_103a.

The translation units are compiled in parallel with nvcc and linked into one
shared library with the C ABI of ``include/bsq.h``.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
OUT = os.path.join(PKG, "_build")
LIB = os.path.join(OUT, "libbsq.so")
SOURCES = ["bsq_kernels.cu", "bsq_host.cu", "bsq_noalloc.cu", "bsq_server.cu"]
HEADERS = ["bsq_internal.cuh", "bsq_launch.h"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# The step kernels compile single-precision sqrt, division and reciprocal to
# the approximate hardware forms (double precision is not affected).
FAST_MATH = ["-use_fast_math"]
FAST_MATH_SOURCES = ["bsq_kernels.cu"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", os.path.join(ROOT, "include")]


def nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libbsq")


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, f) for f in SOURCES + HEADERS] + [os.path.join(ROOT, "include", "bsq.h")]
    return any(os.path.getmtime(p) > t for p in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and not _stale():
        return LIB
    os.makedirs(OUT, exist_ok=True)
    cc = nvcc()
    objs = [os.path.join(OUT, s.replace(".cu", ".o")) for s in SOURCES]

    def compile_one(src, obj):
        extra = FAST_MATH if src in FAST_MATH_SOURCES else []
        cmd = [cc, *ARCH, *FLAGS, *extra, "-c", os.path.join(CSRC, src), "-o", obj]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed on %s:\n%s" % (src, r.stderr))
        return r.stderr

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        logs = list(ex.map(compile_one, SOURCES, objs))
    tmp = LIB + ".%d.tmp" % os.getpid()
    r = subprocess.run([cc, *ARCH, "-shared", *objs, "-o", tmp, "-lcudart"], capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s" % r.stderr)
    os.replace(tmp, LIB)
    if verbose:
        print("\n".join(logs))
    return LIB


if __name__ == "__main__":
    build(force=True, verbose=True)
    print(LIB)
