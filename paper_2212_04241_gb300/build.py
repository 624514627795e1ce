"""Build the GB300 junction-tree library (libjt.so) in-tree.

nvcc compiles the CUDA translation units for sm_103a only; the host
compiler is plain C++17.  The object files are compiled in parallel and
linked into ``_build/libjt.so`` with the CUDA runtime linked statically, so
the library needs nothing from PyTorch at run time.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libjt.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
CUDA_UNITS = ["kernels.cu", "capi.cu", "serve.cu", "noalloc.cu"]
CXX_UNITS = ["compile.cpp", "cpu_layers.cpp"]


def _nvcc() -> str:
    p = shutil.which("nvcc")
    if p:
        return p
    cand = "/usr/local/cuda/bin/nvcc"
    if os.path.exists(cand):
        return cand
    raise RuntimeError("nvcc not found")


def _newest_source_mtime() -> float:
    t = os.path.getmtime(os.path.abspath(__file__))
    for d in (SRC, os.path.join(HERE, "..", "include")):
        for f in os.listdir(d):
            t = max(t, os.path.getmtime(os.path.join(d, f)))
    return t


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= _newest_source_mtime():
        return LIB
    os.makedirs(OUT_DIR, exist_ok=True)
    nvcc = _nvcc()
    tag = f"{os.getpid()}"
    jobs = []
    objs = []
    for u in CUDA_UNITS:
        o = os.path.join(OUT_DIR, u + f".{tag}.o")
        objs.append(o)
        jobs.append([nvcc, *ARCH, "-lineinfo", "-O3", "-std=c++17", "-Xcompiler", "-fPIC",
                     "-Xcompiler", "-fvisibility=hidden", "-c", os.path.join(SRC, u), "-o", o])
    for u in CXX_UNITS:
        o = os.path.join(OUT_DIR, u + f".{tag}.o")
        objs.append(o)
        jobs.append(["g++", "-O2", "-std=c++17", "-fPIC", "-fvisibility=hidden", "-pthread", "-c",
                     os.path.join(SRC, u), "-o", o])

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("build failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
        if verbose and (r.stdout or r.stderr):
            print(r.stdout + r.stderr, file=sys.stderr)

    with cf.ThreadPoolExecutor(max_workers=len(jobs)) as ex:
        list(ex.map(run, jobs))
    tmp = LIB + f".{tag}.tmp"
    run([nvcc, *ARCH, "-shared", "-cudart", "static", "-o", tmp, *objs, "-lpthread"])
    os.replace(tmp, LIB)
    for o in objs:
        os.remove(o)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
