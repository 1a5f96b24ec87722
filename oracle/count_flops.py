"""FP64 operations per cell-update of the method, counted by the op-counting build of the
oracle (opcount.cpp: the oracle compiled with a counting floating-point type).

MEASUREMENT INFRASTRUCTURE, like the oracle: run by hand to write the committed summary
``profiles/fp64_flops_per_cell_update.txt`` that bench.py reads for the FP64 path's ALU
roofline. Usage: python oracle/count_flops.py [--write]

A cell-update is one cell advanced by one full TVD RK2 step of the default scheme:
two stages of (conservative -> primitive, three MUSCL face-state pairs, three HLLC
fluxes (the faces a cell owns), the residual sum, the level-set residual, the stage
update), the wave-speed sum of the next time step, and the reinitialisation amortised
(5 iterations every 10 steps). Each part is counted once per cell or per face, as the
method needs it. FLOPs = additions/subtractions + multiplications + divisions + square
roots (one each); transcendental calls are listed apart. Interface faces (the FIVER
flux: an exact Riemann solve and two fluxes) are counted per face and added with the
interface-face density of the workload.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRC = os.path.join(HERE, "opcount.cpp")
LIB = os.path.join(HERE, "libm2c_opcount.so")
OUT = os.path.join(ROOT, "profiles", "fp64_flops_per_cell_update.txt")

# materials of the 256^3 shock-bubble workload
MG_WATER = (1, [1000.0, 1483.0, 1.75, 0.28, 0.0, -np.inf])
AIR = (0, [1.4, 0.0, 0, 0, 0, 0])
STATES = {
    "water_ambient": (MG_WATER, [1000.0, 0.0, 0.0, 0.0, 1e5]),
    "water_shocked": (MG_WATER, [1243.9677839, 442.83298069, 0.0, 0.0, 1e9]),
    "air": (AIR, [1.2, 0.0, 0.0, 0.0, 1e5]),
}
# volume fractions in the middle of the timed window of bench.py (steps 3..103 of the
# 256^3 workload: the shock, moving 2258 m/s from x = 0.2, is near x = 0.235)
FRACTIONS = {"water_ambient": 0.751, "water_shocked": 0.235, "air": 0.014}
# interface faces per cell in that window (bench.py's interface_faces / cells, about 2.8e4 / 2^24)
IFACE_PER_CELL = 0.0017


def build() -> str:
    if not os.path.exists(LIB) or os.path.getmtime(LIB) < max(os.path.getmtime(SRC),
                                                               os.path.getmtime(os.path.join(HERE, "m2c_oracle.c"))):
        subprocess.run(["g++", "-O1", "-std=c++17", "-fpermissive", "-w", "-ffp-contract=off", "-shared", "-fPIC",
                        "-I", HERE, "-o", LIB, SRC], check=True)
    return LIB


def parts(lib, mat, P):
    out = np.zeros((6, 5))
    prm = np.ascontiguousarray(mat[1], dtype=np.float64)
    st = lib.opc_parts(mat[0], prm.ctypes.data_as(ctypes.c_void_p),
                       np.ascontiguousarray(P, dtype=np.float64).ctypes.data_as(ctypes.c_void_p),
                       out.ctypes.data_as(ctypes.c_void_p))
    assert st == 0
    return out


def per_cell_update(p):
    """FLOPs (add, mul, div, sqrt summed) and special calls of one cell-update."""
    flops = p[:, :4].sum(axis=1)
    spec = p[:, 4]
    stage = flops[0] + 3 * flops[2] + 3 * flops[3] + 45 + 3 * flops[4] + 5
    stage_sp = spec[0] + 3 * spec[2] + 3 * spec[3]
    wave = flops[0] + flops[1] + 1 + 5  # primitive state, c^2, c, sum over three axes
    total = 2 * stage + 12 + 24 + wave + 0.5 * flops[5]
    return total, 2 * stage_sp + spec[0] + spec[1]


def main(write=False):
    lib = ctypes.CDLL(build())
    p = ctypes.c_void_p
    lib.opc_parts.argtypes = [ctypes.c_int, p, p, p]
    lib.opc_fiver_face.argtypes = [ctypes.c_int, p, p, ctypes.c_int, p, p, p, p]
    names = ["cons->prim", "c^2 check", "face-state pair", "HLLC", "level-set derivative", "reinit cell"]
    lines = ["# FP64 operations per cell-update of the default scheme (TVD RK2, modified van Albada, HLLC,",
             "# level set, reinitialisation 5 iterations every 10 steps), counted by the op-counting build",
             "# of the oracle; FLOPs = add/sub + mul + div + sqrt, one each. Command:",
             "#   python oracle/count_flops.py --write", ""]
    per = {}
    for name, (mat, P) in STATES.items():
        cnt = parts(lib, mat, P)
        total, spec = per_cell_update(cnt)
        per[name] = total
        lines.append(f"# {name}: " + ", ".join(f"{n} {int(cnt[k, :4].sum())}" for k, n in enumerate(names)))
        lines.append(f"flops_per_cell_update_{name} = {total:.1f}")
        lines.append(f"special_calls_per_cell_update_{name} = {spec:.1f}")
    iface = []
    # the first face is the quiescent bubble surface of the timed window (the shock has not
    # reached the bubble yet); the others are faces the shock reaches later
    for wL, wR in (((1000.0, 0.0, 1e5), (1.2, 0.0, 1e5)), ((1243.97, 442.83, 1e9), (1.2, 0.0, 1e5)),
                   ((1050.0, 80.0, 2e8), (3.0, 10.0, 4e5))):
        out = np.zeros(5)
        it = ctypes.c_int()
        a = np.ascontiguousarray(MG_WATER[1], dtype=np.float64)
        b = np.ascontiguousarray(AIR[1], dtype=np.float64)
        st = lib.opc_fiver_face(1, a.ctypes.data_as(p), np.array(wL).ctypes.data_as(p), 0, b.ctypes.data_as(p),
                                np.array(wR).ctypes.data_as(p), out.ctypes.data_as(p), ctypes.byref(it))
        assert st == 0
        iface.append(out[:4].sum())
        lines.append(f"# FIVER face water {wL} | air {wR}: {int(out[:4].sum())} flops, {int(out[4])} special, "
                     f"{it.value} iterations")
    fiver = float(iface[0])
    avg = sum(FRACTIONS[k] * per[k] for k in per) + 2 * IFACE_PER_CELL * fiver
    lines += [f"fiver_flops_per_interface_face_quiescent = {fiver:.1f}",
              f"fiver_flops_per_interface_face_shocked = {max(iface[1:]):.1f}",
              f"# workload average in the timed window: volume fractions {FRACTIONS},",
              f"# {IFACE_PER_CELL} quiescent interface faces per cell per stage (two stages per step)",
              f"flops_per_cell_update_256_mg_shock_bubble = {avg:.1f}"]
    text = "\n".join(lines) + "\n"
    print(text)
    if write:
        with open(OUT, "w") as f:
            f.write(text)


if __name__ == "__main__":
    main("--write" in sys.argv)
