"""Build libxorec.so in-tree (paper_2108_02692_gb300/_build/).

Host C++ is compiled with g++, the CUDA executors with nvcc for sm_103a, and
the objects are linked by nvcc into one shared library that exports the C
ABI of include/xorec.h.  Translation units compile in parallel; nothing here
needs a GPU.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
ROOT = os.path.dirname(HERE)
LIB = os.path.join(OUT, "libxorec.so")

CUDA_HOME = os.environ.get("CUDA_HOME", "/usr/local/cuda")
NVCC = os.path.join(CUDA_HOME, "bin", "nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]

HOST_SRCS = ["gf.cc", "slp.cc", "plan.cc", "capi.cc", "jit.cc", "batch.cc", "server.cc", "hostio.cc", "tune.cc"]
CUDA_SRCS = ["executor.cu", "noalloc.cu"]
HEADERS = ["gf.h", "slp.h", "plan.h", "internal.h", "tile_pipeline.cuh"]


def _inputs():
    files = [os.path.join(CSRC, f) for f in HOST_SRCS + CUDA_SRCS + HEADERS]
    files.append(os.path.join(ROOT, "include", "xorec.h"))
    files.append(os.path.abspath(__file__))
    return files


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(f) > t for f in _inputs())


def _run(cmd):
    r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    if r.returncode != 0:
        raise RuntimeError("build step failed:\n" + " ".join(cmd) + "\n" + r.stdout)
    return r.stdout


def _write_pipeline_inc():
    src = open(os.path.join(CSRC, "tile_pipeline.cuh")).read()
    body = 'R"XKSRC(' + src + ')XKSRC"\n'
    path = os.path.join(OUT, "tile_pipeline_src.inc")
    if not os.path.exists(path) or open(path).read() != body:
        with open(path, "w") as f:
            f.write(body)


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and not _stale():
        return LIB
    os.makedirs(OUT, exist_ok=True)
    _write_pipeline_inc()
    inc = ["-I", CSRC, "-I", OUT, "-I", os.path.join(ROOT, "include"),
           "-I", os.path.join(CUDA_HOME, "include")]
    jobs = []
    for f in HOST_SRCS:
        obj = os.path.join(OUT, f + ".o")
        jobs.append(["g++", "-O2", "-std=c++17", "-fPIC", "-Wall", "-Wno-unused-function",
                     *inc, "-c", os.path.join(CSRC, f), "-o", obj])
    for f in CUDA_SRCS:
        obj = os.path.join(OUT, f + ".o")
        jobs.append([NVCC, *ARCH, "-O3", "-lineinfo", "-std=c++17",
                     "-Xcompiler", "-fPIC", "-Xptxas", "-v", *inc, "-c",
                     os.path.join(CSRC, f), "-o", obj])
    with cf.ThreadPoolExecutor(max_workers=len(jobs)) as ex:
        outs = list(ex.map(_run, jobs))
    if verbose:
        for o in outs:
            if o.strip():
                print(o)
    objs = [os.path.join(OUT, f + ".o") for f in HOST_SRCS + CUDA_SRCS]
    tmp = LIB + f".tmp{os.getpid()}"
    _run([NVCC, *ARCH, "-shared", "-o", tmp, *objs,
          "-L", os.path.join(CUDA_HOME, "lib64"), "-lnvrtc",
          "-Xlinker", "-rpath=" + os.path.join(CUDA_HOME, "lib64")])
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
