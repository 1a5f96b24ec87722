"""The op-counting build of the oracle (oracle/opcount.cpp, used for the FP64 path's FLOP
roofline) against hand counts of the stiffened-gas formulas, and its per-cell-update total
against the committed summary. CPU only."""
import os
import shutil

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def counts():
    if shutil.which("g++") is None:
        pytest.skip("no g++")
    from oracle import count_flops as CF
    import ctypes
    lib = ctypes.CDLL(CF.build())
    lib.opc_parts.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    return CF, lib


def test_stiffened_gas_parts_match_hand_counts(counts):
    """cons -> prim for a stiffened gas: u, v, w (3 div), kinetic energy (4 mul, 2 add), e (1 add,
    1 div), p = (g - 1) rho e - g p_c (2 add, 3 mul): 16; c^2 = g (p + p_c)/rho: 3."""
    CF, lib = counts
    c = CF.parts(lib, CF.AIR, [1.2, 3.0, -2.0, 1.0, 1e5])
    assert c[0, :4].sum() == 16 and c[1, :4].sum() == 3
    assert c[0, 2] == 4 and c[1, 2] == 1  # divisions
    assert c[:, 4].sum() == 0  # no transcendental call on the stiffened-gas bulk path


def test_committed_summary_is_current(counts):
    CF, lib = counts
    with open(os.path.join(ROOT, "profiles", "fp64_flops_per_cell_update.txt")) as f:
        vals = dict(line.split(" = ") for line in f if " = " in line and not line.startswith("#"))
    for name, (mat, P) in CF.STATES.items():
        total, _ = CF.per_cell_update(CF.parts(lib, mat, P))
        assert float(vals[f"flops_per_cell_update_{name}"]) == pytest.approx(total, abs=0.05)
