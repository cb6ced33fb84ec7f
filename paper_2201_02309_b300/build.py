"""Build the in-tree CUDA shared library libkatsevich.so for sm_103a."""
from __future__ import annotations

import glob
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
LIBDIR = os.path.join(HERE, "_lib")
LIB = os.path.join(LIBDIR, "libkatsevich.so")
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# simulate.cu: no contraction of multiply-adds, so the FP64 steps that decide a
# random draw round exactly as written (and as the FP64 reference computes them)
EXTRA = {"simulate.cu": ["-fmad=false"]}


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def deps():
    return sources() + sorted(glob.glob(os.path.join(CSRC, "*.cuh"))) + [os.path.join(ROOT, "include", "katsevich.h")]


LIB_DEBUG = os.path.join(LIBDIR, "libkatsevich_debug.so")
# sources whose kernels carry KATS_DEBUG_CHECKS invariant checks (the bounds-checked build)
DEBUG_SOURCES = {"backproject.cu", "backproject_multi.cu"}


def up_to_date(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(d) <= t for d in deps())


def _compile(src: str, obj: str, verbose: bool, defines=()) -> None:
    cmd = [NVCC, "-O3", "-std=c++17", *ARCH, "-lineinfo", "-Xcompiler", "-fPIC,-fvisibility=hidden",
           "-Xptxas", "-v" if verbose else "-O3", *EXTRA.get(os.path.basename(src), []), *defines,
           "-I", os.path.join(ROOT, "include"), "-c", src, "-o", obj]
    subprocess.check_call(cmd)


def _link(lib: str, objs) -> None:
    tmp = lib + f".tmp{os.getpid()}"
    subprocess.check_call([NVCC, "-shared", *ARCH, "-o", tmp, *objs, "-lcudart_static", "-ldl", "-lrt", "-lpthread"])
    os.replace(tmp, lib)


def build(force: bool = False, verbose: bool = False, debug: bool = False) -> str:
    """Compile every .cu under csrc/ into _lib/libkatsevich.so (relocatable device code off).

    debug=True also builds _lib/libkatsevich_debug.so: the same objects, except that the sources
    in DEBUG_SOURCES are compiled with KATS_DEBUG_CHECKS (kernel invariant checks); loaded when
    KATSEVICH_DEBUG_CHECKS=1.  The nvcc calls run in parallel, one per source."""
    from concurrent.futures import ThreadPoolExecutor

    os.makedirs(LIBDIR, exist_ok=True)
    objdir = os.path.join(HERE, "_build")
    dbgdir = os.path.join(HERE, "_build_debug")
    os.makedirs(objdir, exist_ok=True)
    objs = [os.path.join(objdir, os.path.basename(src)[:-3] + ".o") for src in sources()]
    rel = force or not up_to_date(LIB)
    dbg = debug and (force or not up_to_date(LIB_DEBUG))
    jobs = [(src, obj, ()) for src, obj in zip(sources(), objs)] if rel else []
    dobjs = list(objs)
    if dbg:
        os.makedirs(dbgdir, exist_ok=True)
        for i, src in enumerate(sources()):
            if os.path.basename(src) in DEBUG_SOURCES:
                dobjs[i] = os.path.join(dbgdir, os.path.basename(src)[:-3] + ".o")
                jobs.append((src, dobjs[i], ("-DKATS_DEBUG_CHECKS",)))
    if jobs:
        with ThreadPoolExecutor(max_workers=max(1, min(len(jobs), os.cpu_count() or 1))) as pool:
            for f in [pool.submit(_compile, src, obj, verbose, list(defs)) for src, obj, defs in jobs]:
                f.result()  # re-raises a failed compile
    if rel:
        _link(LIB, objs)
    if not debug:
        return LIB
    if dbg:
        _link(LIB_DEBUG, dobjs)
    return LIB_DEBUG


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv, debug="--debug" in sys.argv))
