"""Builds libheom.so in-tree with nvcc for sm_103a (GB300).

Translation units compile in parallel; the shared library links the CUDA
runtime dynamically so it shares one runtime instance with PyTorch.
Usage: ``python -m paper_1012_4382_gb300.build [--force]``.
"""
from __future__ import annotations

import concurrent.futures
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUT = os.path.join(HERE, "libheom.so")
OBJ = os.path.join(HERE, "_build")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
CU_SOURCES = ["heom_kernels_f64_real.cu", "heom_kernels_f64_cplx.cu", "heom_kernels_f32_real.cu",
              "heom_kernels_f32_cplx.cu", "heom_kernels_f32_real_smem.cu", "heom_kernels_f32_cplx_smem.cu",
              "heom_kernels_scaled_f64.cu", "heom_kernels_scaled_f32.cu", "heom_kernels_large.cu",
              "heom_kernels_flow_f32.cu", "heom_kernels_flow_f64.cu", "heom_runtime.cu"]
CPP_SOURCES = ["heom_index.cpp"]


def _nvcc() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found; the CUDA toolkit is required to build libheom")
    return cand


def _sources_newer_than(target: str) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(INCLUDE, "heom.h"), __file__]
    return any(os.path.getmtime(d) > t for d in deps if os.path.isfile(d))


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and not _sources_newer_than(OUT):
        return OUT
    nvcc = _nvcc()
    os.makedirs(OBJ, exist_ok=True)
    common = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-I" + INCLUDE, "-I" + CSRC]
    jobs = []
    for src in CU_SOURCES:
        obj = os.path.join(OBJ, src + ".o")
        jobs.append([nvcc] + ARCH + common + ["-c", os.path.join(CSRC, src), "-o", obj])
    for src in CPP_SOURCES:
        obj = os.path.join(OBJ, src + ".o")
        jobs.append(["g++", "-O2", "-std=c++17", "-fPIC", "-I" + INCLUDE, "-I" + CSRC, "-c",
                     os.path.join(CSRC, src), "-o", obj])

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("build failed:\n%s\n%s%s" % (" ".join(cmd), r.stdout, r.stderr))
        if verbose and (r.stdout or r.stderr):
            sys.stderr.write(r.stdout + r.stderr)

    with concurrent.futures.ThreadPoolExecutor(max_workers=len(jobs)) as ex:
        list(ex.map(run, jobs))
    objs = [os.path.join(OBJ, s + ".o") for s in CU_SOURCES + CPP_SOURCES]
    tmp = OUT + ".tmp%d" % os.getpid()
    run([nvcc] + ARCH + ["-shared", "-cudart", "shared", "-o", tmp] + objs)
    os.replace(tmp, OUT)
    return OUT


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
