"""Builds the GB300 back-end library ``_build/libjdec.so`` (nvcc, sm_103a).

Every translation unit is compiled in parallel for ``sm_103a`` only, with
``-lineinfo``; the objects are linked into one shared library that exports the
C ABI of ``include/jdec.h``.  The CUDA runtime is linked as a shared library.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libjdec.so")
SOURCES = ["jdec_api.cu", "jdec_runtime.cu", "jdec_batch.cu", "jdec_kernels.cu", "jdec_kernels_batch.cu",
           "jdec_entropy.cpp", "jdec_noalloc.cu", "jdec_pipeline.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build the back-end")


def _cuda_home(nvcc: str) -> str:
    return os.path.dirname(os.path.dirname(os.path.realpath(nvcc)))


def _inputs():
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    deps.append(os.path.join(ROOT, "include", "jdec.h"))
    return deps


def _stamp() -> str:
    return os.environ.get("JDEC_EXTRA_NVCC_FLAGS", "")


def build(force: bool = False, verbose: bool = False) -> str:
    stamp_file = LIB + ".flags"
    same_flags = os.path.exists(stamp_file) and open(stamp_file).read() == _stamp()
    if not force and same_flags and os.path.exists(LIB):
        t = os.path.getmtime(LIB)
        if all(os.path.getmtime(d) <= t for d in _inputs()):
            return LIB
    nvcc = _nvcc()
    os.makedirs(BUILD, exist_ok=True)
    flags = ["-std=c++17", "-O3", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-fvisibility=hidden",
             "-diag-suppress", "1160", "-I", os.path.join(ROOT, "include")] + ARCH
    if verbose:
        flags += ["-Xptxas", "-v"]
    # developer knob: extra nvcc flags (e.g. -DJDEC_MIN_CTAS=5), part of the staleness key
    extra = os.environ.get("JDEC_EXTRA_NVCC_FLAGS", "").split()
    flags += extra

    def compile_one(src):
        obj = os.path.join(BUILD, os.path.splitext(src)[0] + ".o")
        cmd = [nvcc] + flags + ["-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
        return obj, r.stderr

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        results = list(ex.map(compile_one, SOURCES))
    if verbose:
        for _, err in results:
            print(err)
    objs = [o for o, _ in results]
    lib64 = os.path.join(_cuda_home(nvcc), "lib64")
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [nvcc] + ARCH + ["-shared", "-cudart", "shared", "-o", tmp] + objs + \
        ["-Xlinker", "-rpath", "-Xlinker", lib64]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    with open(stamp_file, "w") as f:
        f.write(_stamp())
    return LIB


if __name__ == "__main__":
    import sys
    print(build(force="-f" in sys.argv, verbose="-v" in sys.argv))
