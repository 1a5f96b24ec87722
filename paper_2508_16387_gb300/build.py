"""Builds libm2cgpu.so (sm_103a) in the package directory with nvcc."""
from __future__ import annotations

import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SOURCES = [os.path.join(HERE, "csrc", "m2c_solver.cu")]
HEADERS = [os.path.join(HERE, "csrc", f) for f in ("m2c_physics.cuh", "m2c_kernels.cuh")] + \
    [os.path.join(ROOT, "include", "m2c.h")]
LIB = os.path.join(HERE, "libm2cgpu.so")
ARCH = "-gencode=arch=compute_103a,code=sm_103a"


def nvcc_command(out: str = LIB, extra=()):
    return ["nvcc", ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-shared",
            "-I" + os.path.join(ROOT, "include"), "-o", out, *SOURCES, *extra]


def needs_build(out: str = LIB) -> bool:
    if not os.path.exists(out):
        return True
    t = os.path.getmtime(out)
    return any(os.path.getmtime(f) > t for f in SOURCES + HEADERS)


def build(force: bool = False, verbose: bool = False) -> str:
    if force or needs_build():
        cmd = nvcc_command()
        if verbose:
            print(" ".join(cmd))
        subprocess.run(cmd, check=True)
    return LIB


if __name__ == "__main__":
    build(force=True, verbose=True)
