"""Builds the CUDA library libflapw.so in-tree (paper_1712_07206_gb300/_build/).

nvcc for sm_103a only; every translation unit is compiled in parallel, then
linked with the static CUDA runtime.  Host code is compiled with
-ffp-contract=off so that the plane-wave ordering is evaluated exactly as
written.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libflapw.so")
SOURCES = ["api.cu", "gvec.cpp", "ab_gen.cu", "tfactor.cu", "opform.cu", "slicer.cu",
           "herk_f64.cu", "herk_emu.cu", "opgemm.cu", "slegendre.cu", "noalloc.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def _deps():
    files = [os.path.join(SRC, s) for s in SOURCES] + [os.path.join(SRC, "flapw_internal.h"),
                                                       os.path.join(SRC, "tc_common.cuh"),
                                                       os.path.join(SRC, "fixed64.cuh"),
                                                       os.path.join(SRC, "dfloat.cuh"),
                                                       os.path.join(SRC, "alg3.cuh"),
                                                       os.path.join(SRC, "tiles.cuh"),
                                                       os.path.join(ROOT, "include", "flapw.h")]
    return max(os.path.getmtime(f) for f in files)


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= _deps():
        return LIB
    os.makedirs(OUT, exist_ok=True)
    cc = nvcc()
    common = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC,-ffp-contract=off",
              "-I", os.path.join(ROOT, "include"), "-I", SRC] + ARCH

    def compile_one(src):
        obj = os.path.join(OUT, os.path.splitext(src)[0] + ".o")
        cmd = [cc, "-c", os.path.join(SRC, src), "-o", obj] + common
        if src.endswith(".cpp"):
            cmd = [cc, "-x", "c++", "-c", os.path.join(SRC, src), "-o", obj] + common
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        if verbose and (r.stdout or r.stderr):
            print(r.stdout, r.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=min(8, len(SOURCES))) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = LIB + ".tmp%d" % os.getpid()
    cmd = [cc, "-shared", "-o", tmp] + objs + ARCH + ["-cudart", "static", "-lpthread", "-ldl", "-lrt"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
