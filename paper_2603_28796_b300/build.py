"""In-tree build of the native libraries (no JIT cache, no pip install).

- ``libgaloissat.so``: the C-ABI library of ``include/gs.h`` (host loader + sm_103a kernels),
  compiled by nvcc for ``-gencode arch=compute_103a,code=sm_103a``.
- ``libgaloissat_debug.so``: the same sources compiled with ``-DGS_DEBUG``: every row index a
  kernel gathers is checked against the problem's variable count; an index out of range sets a
  sticky status bit (reported by ``gs_sync_status``) and the load is skipped, never trapped.
  Selected at run time by the environment variable ``GS_DEBUG=1``.
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
LIB_DEBUG = os.path.join(HERE, "libgaloissat_debug.so")
SYNTH = os.path.join(HERE, "libgs_synth.so")
BUILD_DIR = os.path.join(HERE, "_build")
BUILD_DIR_DEBUG = os.path.join(HERE, "_build_debug")

CUDA_SOURCES = ["gs_host.cu", "gs_kernels.cu", "gs_st.cu", "gs_pool.cu", "gs_probe.cu", "gs_plan.cpp"]
CUDA_HEADERS = ["gs_internal.h", "gs_plan.h", "gs_device.cuh", "gs_var.cuh", "gs_noise.cuh"]
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


def build_library(force: bool = False, verbose: bool = False, debug: bool = False) -> str:
    lib = LIB_DEBUG if debug else LIB
    build_dir = BUILD_DIR_DEBUG if debug else BUILD_DIR
    srcs = [os.path.join(CSRC, s) for s in CUDA_SOURCES]
    deps = srcs + [os.path.join(CSRC, h) for h in CUDA_HEADERS] + [os.path.join(INCLUDE, "gs.h"), __file__]
    if not force and not _stale(lib, deps):
        return lib
    os.makedirs(build_dir, exist_ok=True)
    nvcc = _nvcc()
    common = [nvcc, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC,
              "-diag-suppress", "177"]
    if debug:
        common += ["-DGS_DEBUG"]
    if verbose:
        common += ["-Xptxas", "-v"]

    def compile_one(src):
        obj = os.path.join(build_dir, os.path.basename(src) + ".o")
        subprocess.run(common + ["-c", src, "-o", obj], check=True)
        return obj

    with ThreadPoolExecutor(max_workers=len(srcs)) as ex:
        objs = list(ex.map(compile_one, srcs))
    tmp = lib + ".tmp%d" % os.getpid()
    subprocess.run([nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-cudart", "static"], check=True)
    os.replace(tmp, lib)
    return lib


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
    with ThreadPoolExecutor(max_workers=2) as ex:
        jobs = [ex.submit(build_library, force, verbose, False), ex.submit(build_library, force, False, True)]
        for j in jobs:
            j.result()


if __name__ == "__main__":
    build_all(force="--force" in sys.argv, verbose="-v" in sys.argv)
    print(LIB)
    print(LIB_DEBUG)
    print(SYNTH)
