"""Build libaf (the CUDA kernels and C ABI) in-tree for sm_103a with nvcc.

The library is written to paper_2506_04857_gb300/_build/libaf.so.  The two
translation units compile in parallel; the whole build takes a few seconds.
"""
from __future__ import annotations

import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libaf.so")
SOURCES = ["af_kernels.cu", "af_adjoint.cu", "af_api.cu", "af_batch.cu", "af_noalloc.cu", "af_api1d.cu"]
HEADERS = ["af_internal.h", "af_math.cuh", "af_device.cuh", "af_kernels1d.cuh"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr"]


def nvcc() -> str:
    path = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(path):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libaf")
    return path


def _stale(out: str, deps) -> bool:
    if not os.path.exists(out):
        return True
    t = os.path.getmtime(out)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile and link libaf.so if any source changed; returns its path."""
    os.makedirs(BUILD, exist_ok=True)
    hdrs = [os.path.join(CSRC, h) for h in HEADERS] + [os.path.join(HERE, "..", "include", "af.h")]
    objs, procs = [], []
    for src in SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(BUILD, src.replace(".cu", ".o"))
        objs.append(o)
        if force or _stale(o, [s] + hdrs):
            cmd = [nvcc(), *ARCH, *FLAGS, "-c", s, "-o", o + ".tmp"]
            if verbose:
                cmd.insert(1, "-Xptxas=-v")
            procs.append((subprocess.Popen(cmd), o))
    failed = False
    for p, o in procs:
        if p.wait() != 0:
            failed = True
        else:
            os.replace(o + ".tmp", o)
    if failed:
        raise RuntimeError("libaf: nvcc compilation failed")
    if force or procs or _stale(LIB, objs):
        tmp = LIB + ".tmp%d" % os.getpid()
        subprocess.check_call([nvcc(), *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"])
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
