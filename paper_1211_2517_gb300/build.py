"""Build the native library ``libkifmm_m2l.so`` in-tree for sm_103a.

Compiles the CUDA sources (nvcc, ``-gencode arch=compute_103a,code=sm_103a``)
and the host C++ sources in parallel into ``_build/`` next to this file,
then links the shared library next to this file.  Rebuilds only what is
out of date.  Usage: ``python -m paper_1211_2517_gb300.build`` or
``paper_1211_2517_gb300.build.build()``.
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
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libkifmm_m2l.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
CUDA_SOURCES = ["api.cu", "batch.cu", "fmm.cu", "kernels_core.cu", "kernels_fmm.cu", "kernels_simt.cu", "kernels_umma.cu", "noalloc.cu",
                "tune.cu"]
CXX_SOURCES = ["precompute.cpp"]
# Per-file flags: the point-source leaf kernels never see subnormal values
# (squared distances in leaf units stay far above 1e-30), so their rsqrtf
# needs no subnormal scaling.
EXTRA_FLAGS = {"kernels_fmm.cu": ["-ftz=true"]}


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libkifmm_m2l.so")


def _headers():
    hs = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".h")]
    return hs + [os.path.join(INCLUDE, "kifmm_m2l.h")]


def _stale(target: str, deps) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def _run(cmd):
    p = subprocess.run(cmd, capture_output=True, text=True)
    if p.returncode != 0:
        raise RuntimeError("build step failed:\n" + " ".join(cmd) + "\n" + p.stdout + p.stderr)
    return p.stdout + p.stderr


def build(verbose: bool = False, ptxas_verbose: bool = False) -> str:
    """Compile and link; returns the path of the shared library."""
    nvcc = _nvcc()
    os.makedirs(BUILD, exist_ok=True)
    hdrs = _headers()
    jobs = []
    objs = []
    for src in CUDA_SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(BUILD, src + ".o")
        objs.append(o)
        if _stale(o, [s, __file__] + hdrs) or ptxas_verbose:
            cmd = [nvcc, *ARCH, "-O3", "-lineinfo", "-std=c++17", *EXTRA_FLAGS.get(src, []), "-Xcompiler", "-fPIC",
                   "-I", INCLUDE, "-c", s, "-o", o]
            if ptxas_verbose:
                cmd.insert(1, "-Xptxas=-v")
            jobs.append(cmd)
    for src in CXX_SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(BUILD, src + ".o")
        objs.append(o)
        if _stale(o, [s, __file__] + hdrs):
            jobs.append([nvcc, "-O3", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-x", "c++",
                         "-c", s, "-o", o])
    if jobs:
        with cf.ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 4)) as ex:
            for out in ex.map(_run, jobs):
                if verbose and out.strip():
                    print(out)
    if _stale(LIB, objs):
        tmp = LIB + ".tmp%d" % os.getpid()
        _run([nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-lpthread"])
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(verbose=True, ptxas_verbose="-v" in sys.argv))
