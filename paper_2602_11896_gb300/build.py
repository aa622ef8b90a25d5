"""Build the in-tree C-ABI library ``libjtfs.so`` for GB300 (sm_103a) with nvcc.

The translation units compile in parallel; the CUDA runtime is linked
statically so the library loads without a GPU (plan inspection works on any
host).  Usage: ``python -m paper_2602_11896_gb300.build`` or ``build()``.
"""

from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(PKG, "libjtfs.so")
SOURCES = ["jtfs_plan.cpp", "jtfs_cuda.cu", "jtfs_batch.cu", "jtfs_decoder.cu", "jtfs_freq_ct_fwd.cu",
           "jtfs_freq_ct_adj.cu", "jtfs_freq_ct_long_fwd.cu",
           "jtfs_freq_ct_long_adj.cu", "jtfs_freq_tc.cu", "jtfs_pool_tc.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libjtfs.so")


def _flags(extra=()):
    return ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O3",
                   "-I", INCLUDE, "-I", CSRC, *extra]


def build(verbose: bool = False, extra_flags=(), out: str = LIB) -> str:
    nvcc = _nvcc()
    bdir = os.path.join(PKG, "_build")
    os.makedirs(bdir, exist_ok=True)

    def compile_one(src: str) -> str:
        obj = os.path.join(bdir, os.path.splitext(src)[0] + ".o")
        cmd = [nvcc, *_flags(extra_flags), "-c", os.path.join(CSRC, src), "-o", obj]
        if src.endswith(".cpp"):
            cmd[1:1] = ["-x", "cu"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        if verbose and (r.stdout or r.stderr):
            print(r.stdout, r.stderr, file=sys.stderr)
        return obj

    with ThreadPoolExecutor(len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = out + ".tmp"
    cmd = [nvcc, *ARCH, "-shared", "-cudart=static", "-o", tmp, *objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, out)
    return out


if __name__ == "__main__":
    print(build(verbose=True))
