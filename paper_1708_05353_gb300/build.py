"""Compile the occ-FMM-K shared library in-tree for sm_103a.

Translation units are compiled in parallel (one nvcc or g++ process each) into
``_build/`` and linked into ``libocck.so`` next to this file.  The host tree
builder is compiled with ``-ffp-contract=off`` so its floating-point decisions
(pair screen, pair centres, box indices) are plain IEEE double expressions.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libocck.so")
CUDA_HOME = os.environ.get("CUDA_HOME", "/usr/local/cuda")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]

CU_SOURCES = ["kernels_ops.cu", "kernels_fmm.cu", "kernels_tc2.cu", "kernels_tc_translate.cu", "kernels_mlp.cu", "kernels_batch.cu", "noalloc.cu", "kernels_f64s.cu"]
CPP_SOURCES = ["host.cpp"]


def _nvcc():
    p = os.path.join(CUDA_HOME, "bin", "nvcc")
    return p if os.path.exists(p) else shutil.which("nvcc")


def _run(cmd):
    r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    if r.returncode != 0:
        raise RuntimeError("build failed:\n" + " ".join(cmd) + "\n" + r.stdout)
    return r.stdout


def _stale(obj, src, deps):
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return any(os.path.getmtime(x) > t for x in [src] + deps)


def build(verbose: bool = False, force: bool = False, ptxas_verbose: bool = False) -> str:
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()
    if nvcc is None:
        raise RuntimeError("nvcc not found")
    headers = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    headers.append(os.path.join(os.path.dirname(HERE), "include", "occk.h"))
    jobs = []
    objs = []
    for f in CU_SOURCES:
        src = os.path.join(CSRC, f)
        if not os.path.exists(src):
            continue
        obj = os.path.join(BUILD, f + ".o")
        objs.append(obj)
        cmd = [nvcc, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
               "--expt-relaxed-constexpr", "-c", src, "-o", obj]
        if ptxas_verbose:
            cmd.insert(1, "-Xptxas=-v")
        if force or _stale(obj, src, headers):
            jobs.append(cmd)
    for f in CPP_SOURCES:
        src = os.path.join(CSRC, f)
        obj = os.path.join(BUILD, f + ".o")
        objs.append(obj)
        cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-ffp-contract=off", "-Wall",
               "-I" + os.path.join(CUDA_HOME, "include"), "-c", src, "-o", obj]
        if force or _stale(obj, src, headers):
            jobs.append(cmd)
    if jobs:
        with ThreadPoolExecutor(max_workers=min(8, len(jobs))) as ex:
            outs = list(ex.map(_run, jobs))
        if verbose:
            for c, o in zip(jobs, outs):
                print(" ".join(c[:2]), "...", c[-1])
                if o.strip():
                    print(o)
    if jobs or not os.path.exists(LIB) or force:
        link = [nvcc, *ARCH, "-shared", "-o", LIB, *objs, "-cudart", "shared",
                "-Xlinker", "-rpath=" + os.path.join(CUDA_HOME, "lib64")]
        _run(link)
    return LIB


if __name__ == "__main__":
    v = "-v" in sys.argv
    print(build(verbose=True, force="--force" in sys.argv, ptxas_verbose=v))
