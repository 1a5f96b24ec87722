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


@pytest.mark.parametrize("left,right,why", [
    ((7, (1.4, 0.0)), (0, (1.4, 0.0)), "left EOS: unknown EOS type"),
    ((0, (1.0, 0.0)), (0, (1.4, 0.0)), "left EOS: SG needs gamma > 1"),
    ((0, (1.4, 0.0)), (1, (1000.0, 1483.0, 0.9, 0.28, 0.0, -float("inf"))), "right EOS: MG needs rho0, c0 > 0, s > 1"),
    ((0, (1.4, 0.0)), (1, (0.0, 1483.0, 1.75, 0.28, 0.0, -float("inf"))), "right EOS: MG needs rho0, c0 > 0, s > 1"),
])
def test_riemann_entry_rejects_bad_eos_before_any_device_work(left, right, why):
    """Argument checks run on the host before any CUDA call, with the reason in
    m2c_last_error(NULL); the EOS rules are those of m2c_set_eos."""
    from paper_2508_16387_gb300 import m2c
    L = m2c.lib()
    eL, eR = m2c.eos_desc(left), m2c.eos_desc(right)
    st = ctypes.c_double * 3
    out = (ctypes.c_double * 4)()
    for fn in (L.m2c_solve_riemann, L.m2c_solve_riemann_mixed):
        code = fn(1, ctypes.byref(eL), st(1.0, 0.0, 1e5), ctypes.byref(eR), st(1.0, 0.0, 1e5), out, None, None, 0,
                  None, 0, None)
        assert code == m2c.M2C_EINVAL
        assert L.m2c_last_error(None).decode().startswith(why)


@pytest.mark.parametrize("n,bc,why", [
    ((1, 1, 1), (0,) * 6, "a grid needs an axis with more than one cell"),
    ((8, 8, 8), (1, 0, 0, 0, 0, 0), "periodic on one side of an axis only"),
    ((8, 8, 8), (3, 3, 0, 0, 0, 0), "unknown boundary condition"),
    ((1, 8, 8), (2, 0, 0, 0, 0, 0), "a symmetry side needs 2 cells along its axis"),
    ((0, 8, 8), (0,) * 6, "grid sizes >= 1"),
])
def test_init_grid_rejects_bad_grids_before_any_device_work(n, bc, why):
    """The grid checks of m2c_init_grid run on the host before the workspace is touched
    (the workspace pointer below is never dereferenced)."""
    from paper_2508_16387_gb300 import m2c
    L = m2c.lib()
    ctx = ctypes.c_void_p()
    code = L.m2c_init_grid(ctypes.byref(ctx), *n, None, 0.1, (ctypes.c_int * 6)(*bc), m2c.FP64,
                           ctypes.c_void_p(256), 1 << 40, None)
    assert code == m2c.M2C_EINVAL and not ctx.value
    assert L.m2c_last_error(None).decode().startswith(why)


def test_binding_raises_with_the_library_text_without_a_context():
    from paper_2508_16387_gb300 import m2c
    L = m2c.lib()
    ctx = ctypes.c_void_p()
    code = L.m2c_init_grid(ctypes.byref(ctx), 1, 1, 1, None, 0.1, (ctypes.c_int * 6)(*(0,) * 6), m2c.FP64,
                           ctypes.c_void_p(256), 1 << 40, None)
    with pytest.raises(m2c.M2CError, match="axis with more than one cell"):
        m2c._check(code, "m2c_init_grid")
    # the next call without a context starts with an empty text
    eos = m2c.eos_desc((m2c.EOS_SG, (1.4, 0.0)))
    out = (ctypes.c_double * 4)()
    st = ctypes.c_double * 3
    assert L.m2c_solve_riemann(0, ctypes.byref(eos), st(), ctypes.byref(eos), st(), out, None, None, 0, None, 0,
                               None) == 0
    assert L.m2c_last_error(None).decode() == ""


def test_context_calls_reject_null_arguments_before_any_device_work():
    """The context entry points return M2C_EINVAL for a null context or null host arrays without
    touching the device (m2c_step_host among them)."""
    from paper_2508_16387_gb300 import m2c
    L = m2c.lib()
    buf = ctypes.c_void_p(256)
    assert L.m2c_step_host(None, buf, buf, 1) == m2c.M2C_EINVAL
    assert L.m2c_step(None, 1) == m2c.M2C_EINVAL
    assert L.m2c_upload_state(None, buf, buf) == m2c.M2C_EINVAL
    assert L.m2c_download_state(None, buf, buf) == m2c.M2C_EINVAL


def test_binding_checks_buffers_before_the_library_sees_them():
    """The binding passes raw pointers, so it checks each buffer's place (host or device),
    type, contiguity and element count first: a wrong buffer raises before any library call."""
    import torch
    from paper_2508_16387_gb300 import m2c
    ok = torch.zeros((5, 2, 3, 4), dtype=torch.float64)
    assert m2c._buf(ok, 120, "W", False).value == ok.data_ptr()
    for bad, err in ((ok.float(), ValueError), (ok[:, :, :, :2], ValueError), (ok.transpose(0, 3), ValueError),
                     (ok.reshape(-1)[:100], ValueError), (ok.numpy(), TypeError)):
        with pytest.raises(err):
            m2c._buf(bad, 120, "W", False)
    with pytest.raises(ValueError, match="device tensor"):
        m2c._buf(ok, 120, "W", True)  # a host tensor where a device buffer is needed
    L = torch.zeros((3, 8), dtype=torch.float64)
    with pytest.raises(ValueError):
        m2c.m2c_solve_riemann((m2c.EOS_SG, (1.4, 0.0)), L, (m2c.EOS_SG, (1.4, 0.0)), L)
    with pytest.raises(ValueError, match=r"\(3, n\)"):
        m2c.m2c_solve_riemann((m2c.EOS_SG, (1.4, 0.0)), L, (m2c.EOS_SG, (1.4, 0.0)), L[:, :4])
    W = torch.zeros((5, 4, 4, 4), dtype=torch.float64)
    phi = torch.zeros((4, 4, 4), dtype=torch.float64)
    with pytest.raises(ValueError):
        m2c.m2c_residual_noalloc((4, 4, 4), 0.25, (0,) * 6, ((0, (1.4, 0.0)), (0, (1.4, 0.0))), W, phi, W, phi)
