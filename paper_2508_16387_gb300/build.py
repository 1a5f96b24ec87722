"""Builds libm2cgpu.so (sm_103a) in the package directory with nvcc."""
from __future__ import annotations

import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SOURCES = [os.path.join(HERE, "csrc", f) for f in ("m2c_solver.cu", "m2c_stage_fp32.cu", "m2c_stage_fp64.cu",
                                                         "m2c_stage_gen.cu")]
HEADERS = [os.path.join(HERE, "csrc", f) for f in ("m2c_physics.cuh", "m2c_riemann.cuh", "m2c_kernels.cuh",
                                                    "m2c_device.cuh", "m2c_stage.cuh", "m2c_stage.h")] + \
    [os.path.join(ROOT, "include", "m2c.h")]
LIB = os.path.join(HERE, "libm2cgpu.so")
ARCH = "-gencode=arch=compute_103a,code=sm_103a"


def nvcc_command(out: str = LIB, extra=()):
    """One nvcc command that compiles and links everything (used by tools that want a single line)."""
    return ["nvcc", ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-shared",
            "-I" + os.path.join(ROOT, "include"), "-o", out, *SOURCES, *extra]


def _compile(src: str, obj: str, extra=()):
    cmd = ["nvcc", ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-c",
           "-I" + os.path.join(ROOT, "include"), "-o", obj, src, *extra]
    subprocess.run(cmd, check=True)
    return obj


def needs_build(out: str = LIB) -> bool:
    if not os.path.exists(out):
        return True
    t = os.path.getmtime(out)
    return any(os.path.getmtime(f) > t for f in SOURCES + HEADERS)


def build(force: bool = False, verbose: bool = False) -> str:
    """Compiles the translation units in parallel, then links the shared library."""
    if force or needs_build():
        from concurrent.futures import ThreadPoolExecutor
        objdir = os.path.join(HERE, "_build")
        os.makedirs(objdir, exist_ok=True)
        objs = [os.path.join(objdir, os.path.basename(f)[:-3] + ".o") for f in SOURCES]
        if verbose:
            print("nvcc -c (parallel):", " ".join(os.path.basename(f) for f in SOURCES))
        with ThreadPoolExecutor(len(SOURCES)) as ex:
            list(ex.map(_compile, SOURCES, objs))
        subprocess.run(["nvcc", ARCH, "-shared", "-o", LIB, *objs], check=True)
    return LIB


if __name__ == "__main__":
    build(force=True, verbose=True)
