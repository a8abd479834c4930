"""Build the CUDA library libbdc.so in-tree (paper_2508_11467_gb300/_build/).

Every csrc/*.cu is compiled for sm_103a only (one -gencode), in parallel, and
linked into one shared library exporting the C ABI of include/bdc.h.  The
data-path sources listed in FP32_SOURCES are compiled a second time with
-DBDC_FP32 (namespace bdc32, single precision) for the *_f32 entry points.  The
CUDA runtime is linked statically so the library does not depend on the
runtime that PyTorch ships.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libbdc.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
CFLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.sep not in cand or os.path.exists(cand)):
            return cand
    return "nvcc"


def _headers_mtime() -> float:
    hs = glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(INCLUDE, "*.h"))
    return max((os.path.getmtime(h) for h in hs), default=0.0)


FP32_SOURCES = ("bdc_driver.cu", "bdc_leaf.cu", "bdc_merge.cu", "bdc_secular.cu", "bdc_gemm64.cu", "bdc_check.cu")


def _compile(job, hdr_mtime: float, force: bool) -> str:
    src, fp32 = job
    obj = os.path.join(BUILD, os.path.basename(src)[:-3] + ("_f32.o" if fp32 else ".o"))
    if (not force and os.path.exists(obj)
            and os.path.getmtime(obj) >= max(os.path.getmtime(src), hdr_mtime)):
        return obj
    tmp = obj + f".{os.getpid()}.tmp"
    cmd = [_nvcc(), *ARCH, *CFLAGS, *(["-DBDC_FP32"] if fp32 else []), "-c", src, "-o", tmp]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, obj)
    return obj


def build(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(BUILD, exist_ok=True)
    srcs = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    jobs = [(s, False) for s in srcs] + [(s, True) for s in srcs if os.path.basename(s) in FP32_SOURCES]
    hdr = _headers_mtime()
    with cf.ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 4)) as ex:
        objs = list(ex.map(lambda j: _compile(j, hdr, force), jobs))
    newest = max(os.path.getmtime(o) for o in objs)
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < newest:
        tmp = LIB + f".{os.getpid()}.tmp"
        cmd = [_nvcc(), *ARCH, "-shared", "-o", tmp, *objs]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, LIB)
    if verbose:
        print(LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True)
