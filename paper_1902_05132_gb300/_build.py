"""Build the CUDA library in-tree (libfmmlayered.so next to this file).

Compiles every translation unit of csrc/ for sm_103a in parallel with nvcc,
then links one shared library exporting the C ABI of include/fmm_layered.h.
"""
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(ROOT, "_build")
LIB = os.path.join(HERE, "libfmmlayered.so")
SOURCES = ["medium.cu", "tree.cu", "ops.cu", "p2p.cu", "api.cu", "noalloc.cu", "m2l_gemm.cu", "m2l_tc.cu", "m2l_rot.cu", "surrogate.cu", "sort.cu", "tables.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-ffp-contract=off",
         "-I" + os.path.join(ROOT, "include")]


def nvcc():
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def _compile(src):
    obj = os.path.join(BUILD, src.replace(".cu", ".o"))
    cmd = [nvcc(), *ARCH, *FLAGS, "-c", os.path.join(CSRC, src), "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stderr}")
    return obj


def build(force=False):
    os.makedirs(BUILD, exist_ok=True)
    newest_src = max(os.path.getmtime(os.path.join(CSRC, f))
                     for f in os.listdir(CSRC)) if os.listdir(CSRC) else 0
    newest_src = max(newest_src, os.path.getmtime(os.path.join(ROOT, "include", "fmm_layered.h")))
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) > newest_src:
        return LIB
    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(_compile, SOURCES))
    cmd = [nvcc(), *ARCH, "-shared", "-o", LIB, *objs, "-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
