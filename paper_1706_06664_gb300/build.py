"""Builds the CUDA library libace_gb300.so in-tree for sm_103a (nvcc, no cmake).

Each translation unit compiles in parallel; the host-side projection generator is built
with g++ and -ffp-contract=off -fno-builtin so its binary64 steps are exactly as written.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIBDIR = os.path.join(HERE, "_lib")
LIB = os.path.join(LIBDIR, "libace_gb300.so")

CU_SOURCES = ["ace_abi.cu", "hash_simt.cu", "hash_tc.cu", "hash_gemm.cu", "tc_probe.cu", "recheck.cu", "count_kernels.cu",
              "exact_score.cu", "hash_fwht.cu"]
CPP_SOURCES = ["projection_gen.cpp"]
HEADERS = ["ace_internal.h", "exact_div.h", "guard.cuh", "tc_ptx.cuh", "tc_plan.h", "gemm_plan.h", "fwht_plan.h",
           "flag_wait.cuh", "score_block.cuh", "f32x2.cuh", "fwht_exact.cuh", "launch_cache.h",
           "admission.h"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def _newer(out: str, deps) -> bool:
    if not os.path.exists(out):
        return False
    t = os.path.getmtime(out)
    return all(os.path.getmtime(d) <= t for d in deps)


def _run(cmd):
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("command failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
    return r.stdout + r.stderr


def build(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(BUILD, exist_ok=True)
    os.makedirs(LIBDIR, exist_ok=True)
    nvcc = _nvcc()
    hdrs = [os.path.join(CSRC, h) for h in HEADERS] + [os.path.join(ROOT, "include", "ace.h")]
    jobs = []
    objs = []
    for src in CU_SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(BUILD, src + ".o")
        objs.append(o)
        if force or not _newer(o, [s] + hdrs):
            jobs.append([nvcc, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-ffp-contract=off",
                         "-Xptxas", "-v", "-I", os.path.join(ROOT, "include"), "-c", s, "-o", o])
    for src in CPP_SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(BUILD, src + ".o")
        objs.append(o)
        if force or not _newer(o, [s] + hdrs):
            cuda_inc = os.path.join(os.path.dirname(os.path.dirname(nvcc)), "include")
            jobs.append(["g++", "-O2", "-fPIC", "-std=c++17", "-ffp-contract=off", "-fno-builtin", "-I", cuda_inc,
                         "-I", os.path.join(ROOT, "include"), "-c", s, "-o", o])
    if jobs:
        with cf.ThreadPoolExecutor(max_workers=min(8, len(jobs))) as ex:
            outs = list(ex.map(_run, jobs))
        if verbose:
            for o in outs:
                sys.stdout.write(o)
        with open(os.path.join(BUILD, "ptxas.log"), "w") as f:
            f.write("\n".join(outs))
    if force or jobs or not _newer(LIB, objs):
        tmp = LIB + f".tmp{os.getpid()}"
        _run([nvcc, *ARCH, "-shared", "-cudart", "static", "-o", tmp, *objs])
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
