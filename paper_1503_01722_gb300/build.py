"""Build the engine's shared library (libocmc.so) from csrc/ with nvcc for sm_103a.

Each .cu file compiles in parallel into _build/, then nvcc links the objects
into libocmc.so next to this file (the CUDA runtime is linked statically).
"""
from __future__ import annotations

import glob
import os
import subprocess
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libocmc.so")
# the checks build: bounds checks on voxel indices, tally addresses and stack slots in the
# transport kernel (a failed check sets an error flag, skips the access, and the call returns
# OCMC_ERR_BOUNDS); same sources, own objects and library
BUILD_CHECKS = os.path.join(HERE, "_build_checks")
LIB_CHECKS = os.path.join(HERE, "libocmc_checks.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", os.path.join(ROOT, "include"), "-I", CSRC]
# FP32 transport code: approximate division/sqrt and flush-to-zero (deterministic for a given
# binary; the physics tables are built in FP64 in ocmc_tables.cu, which keeps IEEE semantics)
# ptxas may fuse a multiply and an add into an FMA differently for different register caps;
# -fmad=false for ptxas keeps the front end's explicit FMAs only, so every compiled variant of
# the transport kernel performs the same arithmetic (bit-identical tallies across launch shapes)
FAST = ["-ftz=true", "-prec-div=false", "-prec-sqrt=false", "-Xptxas", "-fmad=false"]
FAST_FILES = {"ocmc_transport.cu", "ocmc_aux.cu", "ocmc_noalloc.cu"}


def _nvcc():
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.isabs(c) and os.path.exists(c) or not os.path.isabs(c)):
            return c
    return "nvcc"


def _stale(target, deps):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, checks: bool = False) -> str:
    build_dir, lib = (BUILD_CHECKS, LIB_CHECKS) if checks else (BUILD, LIB)
    defs = ["-DOCMC_CHECKS=1"] if checks else []
    srcs = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    headers = [os.path.abspath(__file__)] + glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh")) + \
        glob.glob(os.path.join(ROOT, "include", "*.h"))
    os.makedirs(build_dir, exist_ok=True)
    nvcc = _nvcc()

    def compile_one(src):
        obj = os.path.join(build_dir, os.path.basename(src)[:-3] + ".o")
        if force or _stale(obj, [src] + headers):
            extra = FAST if os.path.basename(src) in FAST_FILES else []
            cmd = [nvcc, *ARCH, *FLAGS, *defs, *extra, "-c", src, "-o", obj + ".tmp"]
            r = subprocess.run(cmd, capture_output=True, text=True)
            if r.returncode != 0:
                raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
            if verbose:
                print(r.stdout, r.stderr)
            os.replace(obj + ".tmp", obj)
        return obj

    with ThreadPoolExecutor(max(1, min(len(srcs), os.cpu_count() or 1))) as ex:
        objs = list(ex.map(compile_one, srcs))
    if force or _stale(lib, objs):
        tmp = lib + f".tmp{os.getpid()}"
        r = subprocess.run([nvcc, *ARCH, "-shared", "-o", tmp, *objs], capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(verbose=True))
