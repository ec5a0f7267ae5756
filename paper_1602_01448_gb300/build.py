"""Compile the CUDA sources into the in-tree shared library ``_lib/libsharp.so``.

nvcc is run once per translation unit, in parallel, for sm_103a only, then
the objects are linked with ``nvcc -shared``.  Objects go to ``_build/``
next to this file (both are ignored by git).
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIBDIR = os.path.join(HERE, "_lib")
LIB = os.path.join(LIBDIR, "libsharp.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
SOURCES = ["raar_128_w0.cu", "raar_128_w1.cu", "raar_64_w0.cu", "raar_64_w1.cu", "frame_kernels_128.cu",
           "frame_kernels_64.cu", "image_kernels.cu", "sharp_api.cu", "noalloc.cu",
           "raar_batch_64_c4.cu", "raar_batch_64_c8.cu", "raar_batch_64_c16.cu",
           "raar_batch_128_c4.cu", "raar_batch_128_c8.cu", "raar_batch_128_c16.cu", "sharp_batch.cu",
           "frame256_ops.cu", "raar_mixed_fp16.cu", "raar_mixed_bf16.cu",
           "raar_mixed256_fp16.cu", "raar_mixed256_bf16.cu", "raar_split256.cu",
           "raar_split256_batch.cu"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _run(cmd):
    p = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    if p.returncode != 0:
        raise RuntimeError("command failed:\n" + " ".join(cmd) + "\n" + p.stdout)
    return p.stdout


def build(verbose: bool = False, ptxas_info: bool = False) -> str:
    os.makedirs(BUILD, exist_ok=True)
    os.makedirs(LIBDIR, exist_ok=True)
    _run([sys.executable, "-c",
          f"import os,runpy; os.chdir({CSRC!r}); runpy.run_path('gen_twiddles.py', run_name='__main__')"])
    cc = nvcc()
    flags = ARCH + ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
                    "--expt-relaxed-constexpr"]
    if ptxas_info:
        flags += ["-Xptxas", "-v"]
    jobs = []
    for src in SOURCES:
        obj = os.path.join(BUILD, src.replace(".cu", ".o"))
        jobs.append([cc] + flags + ["-c", os.path.join(CSRC, src), "-o", obj])
    with cf.ThreadPoolExecutor(max_workers=len(jobs)) as ex:
        outs = list(ex.map(_run, jobs))
    if verbose or ptxas_info:
        for o in outs:
            if o.strip():
                print(o)
    objs = [j[-1] for j in jobs]
    tmp = LIB + ".tmp"
    _run([cc] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcudart"])
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(verbose=True, ptxas_info="-v" in sys.argv))
