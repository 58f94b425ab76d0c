"""Build ``libmwcg.so`` in-tree with nvcc for sm_103a.

One translation unit per arithmetic family plus the host runtime, compiled in
parallel, then linked into a shared library next to this file.  The CUDA
runtime is linked statically (nvcc's default), so the library depends only on
the driver.
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
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libmwcg.so")

SOURCES = ["capi.cu", "batched.cu", "batched_k00.cu", "batched_k01.cu", "batched_k02.cu", "batched_k03.cu",
           "batched_k10.cu", "batched_k11.cu", "batched_k12.cu", "batched_k13.cu", "noalloc.cu", "probe.cu",
           "precond.cu", "inst_fp64.cu", "inst_dw.cu", "inst_qdw.cu", "inst_tw.cu", "inst_qtw.cu", "inst_qw.cu",
           "inst_qqw.cu", "inst_qqf.cu", "inst_qf.cu", "inst_bicg_a.cu", "inst_bicg_b.cu", "inst_bicg_c.cu"]
HEADERS = ["mw_device.cuh", "mw_device4.cuh", "mw_float.cuh", "mw_int.cuh", "cg_kernels.cuh", "cg_float.cuh",
           "bicg_kernels.cuh", "bicg_float.cuh", "batched.cuh", "batched_float.cuh"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "--fmad=false", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
         "-I", INCLUDE, "-I", CSRC]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libmwcg.so")


def _sources():
    return [s for s in SOURCES if os.path.exists(os.path.join(CSRC, s))]


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, s) for s in _sources()]
    deps += [os.path.join(CSRC, h) for h in HEADERS if os.path.exists(os.path.join(CSRC, h))]
    deps += [os.path.join(INCLUDE, "mwcg.h"), os.path.abspath(__file__)]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False) -> str:
    """Compile (if stale) and return the path of libmwcg.so."""
    if not force and not _stale():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    cc = nvcc()
    extra = ["-Xptxas", "-v"] if ptxas_info else []

    def compile_one(src):
        obj = os.path.join(BUILD, os.path.splitext(src)[0] + ".o")
        cmd = [cc, "-c", *ARCH, *FLAGS, *extra, "-o", obj, os.path.join(CSRC, src)]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stderr}")
        return obj, r.stderr

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        results = list(ex.map(compile_one, _sources()))
    if verbose or ptxas_info:
        for obj, err in results:
            if err:
                print(f"--- {os.path.basename(obj)}\n{err}", file=sys.stderr)
    tmp = LIB + f".{os.getpid()}.tmp"
    cmd = [cc, "-shared", *ARCH, "-o", tmp, *[o for o, _ in results]]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, ptxas_info="--ptxas" in sys.argv))
