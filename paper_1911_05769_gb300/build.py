"""Builds the CUDA library ``libat.so`` in-tree for sm_103a with nvcc.

Fifteen translation units (host ABI; FP32 and FP64 single-domain kernels;
FP32 and FP64 ensemble kernels; adjoint kernels; FP32 kernels with FP64
viscous accumulation; single-domain and ensemble FP32 kernels with a
compensated state; blocked synchronous kernels for FP32, FP32 with FP64
viscous accumulation, FP32 ensembles and FP64; scalar 3D kernels; 3D system
kernels) compiled in parallel, one ``-gencode``; static CUDA runtime.
Run as
``python -m paper_1911_05769_gb300.build`` or through ``__graft_entry__.build()``.
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(HERE, "libat.so")
SOURCES = [os.path.join(CSRC, f) for f in (
    "at_api.cu", "at_kernels_f32.cu", "at_kernels_f64.cu", "at_batch_f32.cu", "at_batch_f64.cu", "at_adjoint.cu",
    "at_kernels_f32v.cu", "at_kernels_f32c.cu", "at_batch_f32c.cu", "at_sync_f32.cu", "at_sync_f32v.cu", "at_sync_batch_f32.cu",
    "at_sync_f64.cu", "at_kernels3d.cu", "at_kernels3d_iso.cu", "at_kernels3d_blk.cu", "at_kernels3d_blk32.cu", "at_system3d.cu")]
DEPS = SOURCES + [os.path.join(CSRC, f) for f in ("at_kernels.cuh", "at_device.cuh", "at_adjoint.cuh",
                                                 "at_kernels3d.cuh", "at_kernels3d_blk.cuh")] + [
    os.path.join(INCLUDE, "at.h")]

NVCC_FLAGS = [
    "-O3", "-std=c++17", "-lineinfo",
    "-gencode", "arch=compute_103a,code=sm_103a",
    "-Xcompiler", "-fPIC",
]


def nvcc() -> str:
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def needs_build() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(d) > t for d in DEPS)


def build(force: bool = False, verbose: bool = False) -> str:
    """Compiles every translation unit in parallel, then links libat.so."""
    if not force and not needs_build():
        return LIB
    tag = f"{os.getpid()}"
    objs, procs = [], []
    for src in SOURCES:
        obj = os.path.join(HERE, os.path.basename(src)[:-3] + f".{tag}.o")
        cmd = [nvcc(), *NVCC_FLAGS, "-I", INCLUDE, "-c", src, "-o", obj]
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        procs.append(subprocess.Popen(cmd))
        objs.append(obj)
    rcs = [p.wait() for p in procs]
    try:
        if any(rcs):
            raise subprocess.CalledProcessError(max(rcs), "nvcc")
        tmp = LIB + f".{tag}.tmp"
        cmd = [nvcc(), "-shared", "-gencode", "arch=compute_103a,code=sm_103a", *objs, "-o", tmp]
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        subprocess.check_call(cmd)
        os.replace(tmp, LIB)
    finally:
        for o in objs:
            if os.path.exists(o):
                os.remove(o)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
