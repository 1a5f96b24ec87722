"""The C-ABI library loads and exports every entry point declared in include/m2c.h
(no compute calls: this runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "m2c.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*(m2c_[a-z_]+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("m2c_init_grid", "m2c_set_eos", "m2c_step", "m2c_solve_riemann", "m2c_sync", "m2c_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol():
    from paper_2508_16387_gb300 import build as B
    B.build()
    lib = ctypes.CDLL(B.LIB)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_workspace_size_is_host_only_arithmetic():
    from paper_2508_16387_gb300 import m2c
    n = m2c.m2c_workspace_bytes(64, 64, 64, m2c.FP64)
    assert n > 64 ** 3 * (5 * 8 + 3 * 8) and n % 256 == 0
    assert m2c.m2c_workspace_bytes(0, 1, 1, 0) == 0


def test_binding_fails_loudly_without_the_library(monkeypatch, tmp_path):
    from paper_2508_16387_gb300 import m2c
    monkeypatch.setattr(m2c, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(m2c, "_lib", None)
    with pytest.raises(RuntimeError):
        m2c.lib()
