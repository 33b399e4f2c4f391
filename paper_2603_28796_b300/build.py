"""In-tree build of the native libraries (no JIT cache, no pip install).

- ``libgaloissat.so``: the C-ABI library of ``include/gs.h`` (host loader + sm_103a kernels),
  compiled by nvcc for ``-gencode arch=compute_103a,code=sm_103a``.
- ``libgs_synth.so``: the seeded input generators (plain C, host only).

Both land next to this file so that they travel with the source tree.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(HERE, "libgaloissat.so")
SYNTH = os.path.join(HERE, "libgs_synth.so")
BUILD_DIR = os.path.join(HERE, "_build")

CUDA_SOURCES = ["gs_host.cu", "gs_kernels.cu", "gs_st.cu", "gs_pool.cu", "gs_probe.cu", "gs_plan.cpp"]
CUDA_HEADERS = ["gs_internal.h", "gs_plan.h", "gs_device.cuh", "gs_noise.cuh"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libgaloissat.so")


def _stale(target: str, deps) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build_library(force: bool = False, verbose: bool = False) -> str:
    srcs = [os.path.join(CSRC, s) for s in CUDA_SOURCES]
    deps = srcs + [os.path.join(CSRC, h) for h in CUDA_HEADERS] + [os.path.join(INCLUDE, "gs.h"), __file__]
    if not force and not _stale(LIB, deps):
        return LIB
    os.makedirs(BUILD_DIR, exist_ok=True)
    nvcc = _nvcc()
    common = [nvcc, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC,
              "-diag-suppress", "177"]
    if verbose:
        common += ["-Xptxas", "-v"]

    def compile_one(src):
        obj = os.path.join(BUILD_DIR, os.path.basename(src) + ".o")
        subprocess.run(common + ["-c", src, "-o", obj], check=True)
        return obj

    with ThreadPoolExecutor(max_workers=len(srcs)) as ex:
        objs = list(ex.map(compile_one, srcs))
    tmp = LIB + ".tmp%d" % os.getpid()
    subprocess.run([nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-cudart", "static"], check=True)
    os.replace(tmp, LIB)
    return LIB


def build_synth(force: bool = False) -> str:
    src = os.path.join(CSRC, "synth.c")
    if not force and not _stale(SYNTH, [src, __file__]):
        return SYNTH
    tmp = SYNTH + ".tmp%d" % os.getpid()
    subprocess.run(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", src, "-o", tmp, "-lm"], check=True)
    os.replace(tmp, SYNTH)
    return SYNTH


def build_all(force: bool = False, verbose: bool = False) -> None:
    build_synth(force)
    build_library(force, verbose)


if __name__ == "__main__":
    build_all(force="--force" in sys.argv, verbose="-v" in sys.argv)
    print(LIB)
    print(SYNTH)
