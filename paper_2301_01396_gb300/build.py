"""Compiles the sm_103a CUDA library ``_lib/libdiffxpbd.so`` in-tree with nvcc.

Each translation unit is compiled in parallel, then linked into one shared object that
exports the C ABI of ``include/diffxpbd.h``."""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_lib")
LIB_PATH = os.path.join(OUT_DIR, "libdiffxpbd.so")
SOURCES = ["xpbd_kernels.cu", "xpbd_phase.cu", "xpbd_implicit.cu", "xpbd_api.cu", "xpbd_serve.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# Division and square root use the approximate hardware forms (about 1 ulp): the kernels
# are latency-bound and the IEEE sequences lengthen every constraint's dependency chain;
# the parity bounds of the tests hold with them.
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-prec-div=false", "-prec-sqrt=false", "-Xcompiler", "-fPIC",
         "-Xcompiler", "-O2"]


def nvcc() -> str:
    exe = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(exe):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build the library")
    return exe


def _deps() -> list:
    inc = os.path.join(os.path.dirname(HERE), "include", "diffxpbd.h")
    return [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [inc, os.path.abspath(__file__)]


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False) -> str:
    os.makedirs(OUT_DIR, exist_ok=True)
    if not force and os.path.exists(LIB_PATH):
        t = os.path.getmtime(LIB_PATH)
        if all(os.path.getmtime(d) <= t for d in _deps()):
            return LIB_PATH
    exe = nvcc()
    extra = ["-Xptxas", "-v"] if ptxas_info else []

    def compile_one(src):
        obj = os.path.join(OUT_DIR, src.replace(".cu", ".o"))
        cmd = [exe, *ARCH, *FLAGS, *extra, "-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stderr}")
        return obj, r.stderr

    with cf.ThreadPoolExecutor(len(SOURCES)) as ex:
        results = list(ex.map(compile_one, SOURCES))
    if verbose or ptxas_info:
        for _, err in results:
            print(err)
    tmp = LIB_PATH + f".tmp{os.getpid()}"
    cmd = [exe, *ARCH, "-shared", "-o", tmp, *[o for o, _ in results]]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc link failed:\n{r.stderr}")
    os.replace(tmp, LIB_PATH)
    return LIB_PATH


if __name__ == "__main__":
    import sys
    print(build(force=True, ptxas_info="-v" in sys.argv))
