"""Builds libgevo.so (the C ABI of include/gevo.h) in-tree with nvcc for sm_103a.

Each translation unit is compiled in parallel, then linked with -shared; the
result lands next to this file and is git-ignored.  No torch extension
machinery is involved: the library exports plain `extern "C"` symbols.
A second, measurement-only library, libgevo_probes.so (include/gevo_bench.h:
FP32 FMA and ex2 throughput probes that bench.py uses to check the derived
peaks), is built the same way and is not part of libgevo.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
ROOT = os.path.dirname(HERE)
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libgevo.so")
SOURCES = ["api.cu", "project.cu", "binsort.cu", "render.cu", "loss.cu", "active.cu", "optim.cu", "gemm_tc.cu", "unet.cu", "init.cu"]
PROBE_LIB = os.path.join(HERE, "libgevo_probes.so")
PROBE_SOURCES = ["peaks.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE,
              "--expt-relaxed-constexpr"]


def _nvcc():
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def _deps():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + \
        [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE)]
    return max(os.path.getmtime(f) for f in files)


def up_to_date() -> bool:
    return all(os.path.exists(p) and os.path.getmtime(p) >= _deps() for p in (LIB, PROBE_LIB))


def build(force: bool = False, verbose: bool = False, extra_flags=()) -> str:
    """Builds both libraries (if stale) and returns the path of libgevo.so."""
    if not force and up_to_date():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()

    def compile_one(src):
        obj = os.path.join(BUILD, src.replace(".cu", ".o"))
        cmd = [nvcc, *ARCH, *NVCC_FLAGS, *extra_flags, "-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
        if verbose and (r.stdout or r.stderr):
            print(r.stdout, r.stderr, file=sys.stderr)
        return obj

    def link(objs, out):
        tmp = out + f".tmp{os.getpid()}"
        cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, out)

    srcs = SOURCES + PROBE_SOURCES
    with cf.ThreadPoolExecutor(max_workers=len(srcs)) as ex:
        objs = dict(zip(srcs, ex.map(compile_one, srcs)))
    link([objs[s] for s in SOURCES], LIB)
    link([objs[s] for s in PROBE_SOURCES], PROBE_LIB)
    return LIB


if __name__ == "__main__":
    force = "--force" in sys.argv
    print(build(force=force, verbose=True))
