"""Build libmslam.so (sm_103a) in-tree with nvcc.

Each CUDA translation unit is compiled in parallel to an object file, then
linked into one shared library under ``paper_2412_12392_gb300/_build``.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libmslam.so")
SOURCES = ["plan.cu", "match.cu", "linearize.cu", "solve.cu", "backward.cu", "noalloc.cu", "fuse.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA 13 toolkit is required to build libmslam.so")


def _flags(extra=()):
    return ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
                   "-I", os.path.join(HERE, "..", "include")] + list(extra)


def build_variant(out_dir: str, defines=()) -> str:
    """Build a copy of the library with extra -D tuning macros into out_dir
    (used by tuning sweeps; the default build uses the macros' defaults)."""
    os.makedirs(out_dir, exist_ok=True)
    nv = nvcc()
    dflags = [f"-D{d}" for d in defines]
    objs = []

    def one(src):
        o = os.path.join(out_dir, src.replace(".cu", ".o"))
        r = subprocess.run([nv, "-c", os.path.join(CSRC, src), "-o", o] + _flags(dflags), capture_output=True,
                           text=True)
        if r.returncode != 0:
            raise RuntimeError(r.stderr)
        return o

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(one, SOURCES))
    lib = os.path.join(out_dir, "libmslam.so")
    r = subprocess.run([nv, "-shared", "-o", lib] + objs + ARCH, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(r.stderr)
    return lib


def _stale(obj: str, src: str) -> bool:
    if not os.path.exists(obj):
        return True
    deps = [src, os.path.join(CSRC, "common.cuh"), os.path.join(HERE, "..", "include", "mslam.h")]
    return os.path.getmtime(obj) < max(os.path.getmtime(d) for d in deps)


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False) -> str:
    os.makedirs(BUILD, exist_ok=True)
    nv = nvcc()
    jobs = []
    for src in SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(BUILD, src.replace(".cu", ".o"))
        if force or ptxas_info or _stale(o, s):
            extra = ["-Xptxas", "-v"] if ptxas_info else []
            jobs.append(([nv, "-c", s, "-o", o] + _flags(extra), src))

    def run(cmd_src):
        cmd, src = cmd_src
        r = subprocess.run(cmd, capture_output=True, text=True)
        return src, r

    with cf.ThreadPoolExecutor(max_workers=len(jobs) or 1) as ex:
        for src, r in ex.map(run, jobs):
            if verbose or ptxas_info or r.returncode != 0:
                sys.stderr.write(f"--- {src}\n{r.stdout}{r.stderr}")
            if r.returncode != 0:
                raise RuntimeError(f"nvcc failed for {src}")
    objs = [os.path.join(BUILD, s.replace(".cu", ".o")) for s in SOURCES]
    if force or jobs or not os.path.exists(LIB):
        tmp = LIB + f".tmp{os.getpid()}"
        r = subprocess.run([nv, "-shared", "-o", tmp] + objs + ARCH, capture_output=True, text=True)
        if r.returncode != 0:
            sys.stderr.write(r.stdout + r.stderr)
            raise RuntimeError("link of libmslam.so failed")
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True, ptxas_info="--ptxas" in sys.argv)
    print(LIB)
