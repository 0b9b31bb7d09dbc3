"""Compile the CUDA/C++ sources of the TPCG library into an in-tree shared library for sm_103a.

The library is built next to this file (``libtpcg_gb300.so``); objects go to ``_build/``.  nvcc compiles
for ``-gencode arch=compute_103a,code=sm_103a`` only; translation units are compiled in parallel.
"""
from __future__ import annotations

import concurrent.futures as cf
import hashlib
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OBJ = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libtpcg_gb300.so")
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
CU_SOURCES = ["round.cu", "eig.cu", "ops.cu", "api.cu", "elast.cu", "prof.cu", "dst.cu", "gemm_tc.cu"]
CXX_SOURCES = ["setup.cpp", "expsum.cpp"]


def _digest() -> str:
    h = hashlib.sha256()
    for d in (CSRC, os.path.join(ROOT, "include")):
        for f in sorted(os.listdir(d)):
            p = os.path.join(d, f)
            if os.path.isfile(p):
                h.update(f.encode())
                with open(p, "rb") as fh:
                    h.update(fh.read())
    h.update(" ".join(ARCH).encode())
    return h.hexdigest()[:16]


def _run(cmd):
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("build failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
    return r.stdout + r.stderr


def build(force: bool = False, verbose: bool = False) -> str:
    """Build (if sources changed) and return the path of the shared library."""
    os.makedirs(OBJ, exist_ok=True)
    stamp = os.path.join(OBJ, "stamp")
    dig = _digest()
    if not force and os.path.exists(LIB) and os.path.exists(stamp) and open(stamp).read() == dig:
        return LIB
    common = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-I" + os.path.join(ROOT, "include")]
    jobs = []
    for s in CU_SOURCES:
        if not os.path.exists(os.path.join(CSRC, s)):
            continue
        jobs.append([NVCC, *ARCH, *common, "-c", os.path.join(CSRC, s), "-o", os.path.join(OBJ, s + ".o")])
    for s in CXX_SOURCES:
        jobs.append([NVCC, *common, "-x", "c++", "-c", os.path.join(CSRC, s), "-o", os.path.join(OBJ, s + ".o")])
    with cf.ThreadPoolExecutor(max_workers=len(jobs)) as ex:
        outs = list(ex.map(_run, jobs))
    if verbose:
        for o in outs:
            if o.strip():
                print(o)
    objs = [j[-1] for j in jobs]
    tmp = LIB + ".tmp"
    _run([NVCC, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"])
    os.replace(tmp, LIB)
    with open(stamp, "w") as fh:
        fh.write(dig)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
