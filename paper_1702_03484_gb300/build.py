"""Build libmapsq.so (CUDA for sm_103a) in-tree, and libmapsq_checked.so, the
same sources with device bounds checks (-DMAPSQ_CHECKED).

Each translation unit of both libraries is compiled by nvcc in parallel, then
linked into one shared library each, next to this file.  No CMake; a minute or
two on a cold cache.
"""
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
BUILD = os.path.join(ROOT, "_build")
LIB = os.path.join(PKG, "libmapsq.so")
LIB_CHECKED = os.path.join(PKG, "libmapsq_checked.so")

SOURCES = ["api.cu", "prim.cu", "store.cu", "scan.cu", "join.cu", "query.cu", "serve.cu", "autotune.cu", "select.cu", "star.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def flags(extra=()):
    return ARCH + ["-O3", "-std=c++17", "-lineinfo", "--expt-relaxed-constexpr", "-Xcompiler", "-fPIC", "-Xcompiler", "-fvisibility=hidden",
                   "-I", INCLUDE, "-I", CSRC] + list(extra)


def _newer(target: str, deps) -> bool:
    if not os.path.exists(target):
        return False
    t = os.path.getmtime(target)
    return all(os.path.getmtime(d) <= t for d in deps)


def build(verbose: bool = False, extra=()) -> str:
    os.makedirs(BUILD, exist_ok=True)
    headers = [os.path.join(CSRC, h) for h in os.listdir(CSRC) if h.endswith((".cuh", ".h"))]
    headers.append(os.path.join(INCLUDE, "mapsq.h"))
    cc = nvcc()
    variants = [(LIB, BUILD, list(extra)), (LIB_CHECKED, os.path.join(BUILD, "checked"), list(extra) + ["-DMAPSQ_CHECKED"])]
    jobs, links = [], []
    for lib, obj_dir, fl in variants:
        os.makedirs(obj_dir, exist_ok=True)
        objs = []
        for src in SOURCES:
            s = os.path.join(CSRC, src)
            o = os.path.join(obj_dir, src.replace(".cu", ".o"))
            objs.append(o)
            if not _newer(o, [s, __file__] + headers):
                jobs.append([cc] + flags(fl) + ["-c", s, "-o", o])
        links.append((lib, objs))

    def run(cmd):
        if verbose:
            print(" ".join(cmd), flush=True)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed:\n{' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
        return r.stderr

    with cf.ThreadPoolExecutor(max_workers=max(1, min(len(jobs), os.cpu_count() or 4))) as ex:
        for msg in ex.map(run, jobs):
            if verbose and msg:
                print(msg, file=sys.stderr)
    for lib, objs in links:
        if not _newer(lib, objs):
            tmp = lib + ".tmp"
            run([cc] + ARCH + ["-shared", "-o", tmp] + objs)
            os.replace(tmp, lib)
    return LIB


if __name__ == "__main__":
    print(build(verbose=True))
