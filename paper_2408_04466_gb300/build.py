"""Build libgwn.so (CUDA kernels + C ABI) for sm_103a, in-tree.

Each translation unit is compiled by nvcc in parallel, then linked into
``paper_2408_04466_gb300/_build/libgwn.so``.  Usage: ``python -m
paper_2408_04466_gb300.build`` (or ``build()`` from Python).  Set
GWN_NVCC_EXTRA for extra flags (e.g. "-Xptxas -v").
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shlex
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libgwn.so")
SOURCES = ["api.cpp", "bterm.cu", "traverse.cu", "bvh.cu", "backward.cu", "brute.cu", "bezier2d.cu", "batch.cu", "noalloc.cu", "patches.cu", "meshbatch.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def _flags():
    f = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O2,-fvisibility=hidden",
                "--expt-relaxed-constexpr", "-I", os.path.join(HERE, "..", "include")]
    extra = os.environ.get("GWN_NVCC_EXTRA")
    if extra:
        f += shlex.split(extra)
    return f


def _compile(src: str) -> str:
    obj = os.path.join(OUT, os.path.basename(src) + ".o")
    cmd = [nvcc()] + _flags() + ["-x", "cu" if src.endswith(".cu") else "c++", "-c",
                                 os.path.join(SRC, src), "-o", obj]
    if src.endswith(".cpp"):
        cmd = [nvcc()] + _flags() + ["-c", os.path.join(SRC, src), "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
    if r.stderr.strip():
        sys.stderr.write(r.stderr)
    return obj


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(SRC, f) for f in os.listdir(SRC)] + [os.path.join(HERE, "..", "include", "gwn.h"),
                                                              os.path.abspath(__file__)]
    return any(os.path.getmtime(p) > t for p in deps if os.path.exists(p))


def build(force: bool = False, jobs: int | None = None) -> str:
    os.makedirs(OUT, exist_ok=True)
    if not force and not _stale():
        return LIB
    jobs = jobs or min(len(SOURCES), max(1, os.cpu_count() or 1))
    with cf.ThreadPoolExecutor(jobs) as ex:
        objs = list(ex.map(_compile, SOURCES))
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [nvcc()] + ARCH + ["-shared", "-cudart", "shared", "-o", tmp] + objs
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
