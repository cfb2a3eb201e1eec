"""Build ``liblbdp.so`` in-tree for sm_103a (GB300).

Each translation unit under ``csrc/`` compiles in parallel to an object with
``nvcc -gencode arch=compute_103a,code=sm_103a -lineinfo``; the objects link
into ``_build/liblbdp.so``.  Nothing is installed: the Python binding loads the
library from this directory.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(PKG, "csrc")
INC = os.path.join(os.path.dirname(PKG), "include")
OUT = os.path.join(PKG, "_build")
LIB = os.path.join(OUT, "liblbdp.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
         "-I", SRC, "-I", INC]


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build liblbdp")


def _stale(target: str, deps) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, extra=()) -> str:
    nvcc = _nvcc()
    os.makedirs(OUT, exist_ok=True)
    units = sorted(glob.glob(os.path.join(SRC, "*.cu")))
    headers = (glob.glob(os.path.join(SRC, "*.cuh")) + glob.glob(os.path.join(SRC, "*.h"))
               + glob.glob(os.path.join(INC, "*.h")))
    objs = []
    jobs = []
    for u in units:
        o = os.path.join(OUT, os.path.basename(u)[:-3] + ".o")
        objs.append(o)
        if force or _stale(o, [u] + headers):
            jobs.append([nvcc, *ARCH, *FLAGS, *extra, "-c", u, "-o", o])
    if jobs:
        with cf.ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 4)) as ex:
            results = list(ex.map(lambda c: subprocess.run(c, capture_output=True, text=True), jobs))
        for cmd, r in zip(jobs, results):
            if verbose and r.stderr:
                sys.stderr.write(r.stderr)
            if r.returncode != 0:
                sys.stderr.write(r.stdout + r.stderr)
                raise RuntimeError("nvcc failed: " + " ".join(cmd))
    if force or jobs or _stale(LIB, objs):
        tmp = LIB + ".tmp%d" % os.getpid()
        r = subprocess.run([nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"],
                           capture_output=True, text=True)
        if r.returncode != 0:
            sys.stderr.write(r.stdout + r.stderr)
            raise RuntimeError("link of liblbdp.so failed")
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
