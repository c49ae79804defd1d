"""Build libfewha.so in-tree for sm_103a (B300) with nvcc / g++.

    python -m paper_2009_00946_b300.build [--force] [--release-only]

Host setup code is compiled by g++ with FP contraction off (the FP64 geometry
tables are then evaluated exactly as written); CUDA sources by nvcc for
compute_103a / sm_103a.  The library links the CUDA runtime dynamically.

Two variants are built from the same sources, their objects compiled in
parallel: the release library libfewha.so and the debug library
libfewha_debug.so (-DFEWHA_DEBUG: bounds checks at every gather and scatter
of the hot path, reported by fewha_debug_bounds; loaded instead of the
release library when the environment sets FEWHA_DEBUG=1).
"""

from __future__ import annotations

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libfewha.so")
BUILD_DEBUG = os.path.join(HERE, "_build_debug")
LIB_DEBUG = os.path.join(HERE, "libfewha_debug.so")
# variant: (object folder, library, extra defines)
VARIANTS = {"release": (BUILD, LIB, []), "debug": (BUILD_DEBUG, LIB_DEBUG, ["-DFEWHA_DEBUG"])}
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]

CU_SOURCES = ["solver.cu", "fused.cu", "fitcg.cu", "noalloc.cu", "l2bw.cu"]
CPP_SOURCES = ["setup.cpp", "api.cpp"]
# every header of csrc/ is a dependency of every object (a conservative rule:
# an edited header rebuilds all objects)
HEADERS = sorted(f for f in os.listdir(CSRC) if f.endswith((".h", ".cuh")))


def _newer(target: str, deps: list[str]) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def _run(cmd: list[str]) -> None:
    print(" ".join(cmd), flush=True)
    subprocess.run(cmd, check=True)


def build(force: bool = False, verbose_ptxas: bool = False, variants=("release", "debug")) -> str:
    hdrs = [os.path.join(CSRC, h) for h in HEADERS] + [os.path.join(INCLUDE, "fewha.h")]
    compiles, links = [], []
    for v in variants:
        bdir, lib, defs = VARIANTS[v]
        os.makedirs(bdir, exist_ok=True)
        objs = []
        for src in CPP_SOURCES:
            s = os.path.join(CSRC, src)
            o = os.path.join(bdir, src + ".o")
            objs.append(o)
            if force or _newer(o, [s] + hdrs):
                compiles.append(["g++", "-std=c++17", "-O2", "-fPIC", "-ffp-contract=off", "-Wall",
                                 "-Wno-unused-variable"] + defs +
                                ["-I", INCLUDE, "-I", CSRC, "-I", "/usr/local/cuda/include", "-c", s, "-o", o])
        for src in CU_SOURCES:
            s = os.path.join(CSRC, src)
            o = os.path.join(bdir, src + ".o")
            objs.append(o)
            if force or _newer(o, [s] + hdrs):
                cmd = [NVCC] + ARCH + ["-std=c++17", "-O3", "-lineinfo", "-Xcompiler", "-fPIC",
                                       "--expt-relaxed-constexpr"] + defs + ["-I", INCLUDE, "-I", CSRC, "-c", s, "-o", o]
                if verbose_ptxas:
                    cmd.insert(1, "-Xptxas=-v")
                compiles.append(cmd)
        links.append((lib, objs))
    if compiles:
        workers = max(1, min(len(compiles), os.cpu_count() or 1))
        with ThreadPoolExecutor(workers) as pool:
            for f in [pool.submit(_run, c) for c in compiles]:
                f.result()   # raises CalledProcessError of a failed compile
    for lib, objs in links:
        if force or _newer(lib, objs):
            _run([NVCC] + ARCH + ["-shared", "-cudart", "shared", "-o", lib] + objs +
                 ["-Xlinker", "-rpath,/usr/local/cuda/lib64"])
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose_ptxas="--ptxas-v" in sys.argv,
          variants=("release",) if "--release-only" in sys.argv else ("release", "debug"))
