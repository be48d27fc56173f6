"""Build liblbe.so (the CUDA C-ABI library) in-tree with nvcc for sm_103a.

Each translation unit compiles in parallel; the FP64 step kernel and the
state kernels are compiled without FMA contraction, so that FP64 mode rounds
operation by operation like the FP64 CPU reference.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "liblbe.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I" + INCLUDE]
UNITS = {
    "lbe_step_f64.cu": ["-fmad=false"],
    # FP32 arithmetic: division and square root to within 2 ulp (a few
    # instructions instead of the IEEE-rounded sequences)
    "lbe_step_f32.cu": ["-prec-div=false", "-prec-sqrt=false"],
    "lbe_step_f16.cu": ["-prec-div=false", "-prec-sqrt=false"],
    "lbe_step_bf16.cu": ["-prec-div=false", "-prec-sqrt=false"],
    "lbe_step_mix.cu": ["-prec-div=false", "-prec-sqrt=false"],
    "lbe_aux.cu": ["-fmad=false"],
    "lbe_api.cu": ["-Xcompiler", "-ffp-contract=off"],
    "lbe_noalloc.cu": ["-fmad=false"],
    "lbe_adjoint.cu": [],
}


def nvcc() -> str:
    p = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(p):
        raise RuntimeError("nvcc not found: the CUDA library cannot be built")
    return p


def _sources():
    return [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(INCLUDE, "lbe.h")]


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(s) <= t for s in _sources())


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and up_to_date():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    nv = nvcc()

    def one(unit):
        src = os.path.join(CSRC, unit)
        obj = os.path.join(BUILD, unit.replace(".cu", ".o"))
        cmd = [nv] + ARCH + FLAGS + UNITS[unit] + ["-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (unit, " ".join(cmd), r.stderr))
        if verbose and r.stderr:
            print(r.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=len(UNITS)) as ex:
        objs = list(ex.map(one, UNITS))
    tmp = LIB + ".%d.tmp" % os.getpid()
    cmd = [nv] + ARCH + ["-shared", "-o", tmp] + objs
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s\n%s" % (" ".join(cmd), r.stderr))
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
