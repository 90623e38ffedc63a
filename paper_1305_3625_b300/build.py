"""Build the CUDA library libfftconv.so in-tree for sm_103a (B300).

nvcc cross-compiles without a GPU.  The shared library is placed next to this
file so that it travels with the source tree.  The translation units (the
library, the server and one unit per padded FFT size holding that size's pass
kernels) compile in parallel into _build/ and are then linked.
"""
from __future__ import annotations

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libfftconv.so")
OBJDIR = os.path.join(HERE, "_build")
SOURCES = ["fc_lib.cu", "fc_server.cu", "fc_var_small.cu", "fc_var_256.cu", "fc_var_512.cu", "fc_var_1024.cu",
           "fc_var_2048.cu", "fc_var_4096.cu", "fc_var_8192.cu"]
HEADERS = ["fc_fft.cuh", "fc_passes.cuh", "fc_internal.h", "fc_persist.cuh", "fc_tma.cuh", "fc_variants.h",
           "fc_variants.cuh", "fc_alloc.h"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr"]


def _inputs():
    root = os.path.dirname(HERE)
    files = [os.path.join(CSRC, f) for f in SOURCES + HEADERS]
    files.append(os.path.join(root, "include", "fftconv.h"))
    return files


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(f) <= t for f in _inputs())


def _compile(nvcc: str, src: str, verbose: bool, force: bool) -> str:
    obj = os.path.join(OBJDIR, os.path.splitext(src)[0] + ".o")
    deps = [os.path.join(CSRC, src)] + [f for f in _inputs() if not f.endswith(".cu")]
    if not force and os.path.exists(obj) and all(os.path.getmtime(f) <= os.path.getmtime(obj) for f in deps):
        return obj
    cmd = [nvcc, *NVCC_FLAGS, "-c", "-o", obj, os.path.join(CSRC, src)]
    if verbose:
        print(" ".join(cmd), file=sys.stderr)
    subprocess.run(cmd, check=True)
    return obj


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and up_to_date():
        return LIB
    nvcc = os.environ.get("NVCC", "nvcc")
    os.makedirs(OBJDIR, exist_ok=True)
    jobs = int(os.environ.get("FC_BUILD_JOBS", str(os.cpu_count() or 1)))
    with ThreadPoolExecutor(max_workers=max(1, jobs)) as ex:
        objs = list(ex.map(lambda f: _compile(nvcc, f, verbose, force), SOURCES))
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *objs]
    if verbose:
        print(" ".join(cmd), file=sys.stderr)
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
