"""The allocation-free residual entry point against the context entry point.

m2c_residual_noalloc serves callers that cannot allocate device memory (their
device memory comes from a fixed pool they do not own, or they must not cause
the device-wide synchronisation of cudaMalloc/cudaFree): it computes the stage
residual with its scratch in one library-held device array. This file is
collected last so that a run stopping at its first failure has already run
every other test; it passes alone in a fresh process and after the others.
"""
import ctypes

import numpy as np
import pytest

from paper_2508_16387_gb300 import workloads as WL


@pytest.fixture(scope="module")
def m2c():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2508_16387_gb300 import m2c as M
    M.lib()
    return M


def _case(M, n, seed, water, precision):
    import torch
    P, phi = WL.random_state(n, seed=seed, eos=(water, WL.AIR_PG), two_phase=True)
    bc = (0, 0, 1, 1, 0, 0)
    g = M.Grid(n, 1.0 / n[0], bc, (water, WL.AIR_PG), precision=precision)
    g.set_prims(P, phi)
    R_ctx, L_ctx = g.residual()
    W = g.W.clone()
    ph = g.phi.clone()
    R = torch.full_like(R_ctx, float("nan"))
    L = torch.full_like(L_ctx, float("nan"))
    code = M.m2c_residual_noalloc(n, 1.0 / n[0], bc, (water, WL.AIR_PG), W, ph, R, L, precision=precision)
    torch.cuda.synchronize()
    return code, R.cpu().numpy(), L.cpu().numpy(), R_ctx.cpu().numpy(), L_ctx.cpu().numpy()


@pytest.mark.gpu
def test_noalloc_residual_matches_context_residual_twice_in_a_row(m2c):
    # two calls in a row on different grids and materials: the second call must not see the
    # first call's counters or lists, which stay in the shared array
    for n, seed, water, prec in (((40, 24, 20), 3, WL.WATER_SG, m2c.FP64),
                                 ((33, 17, 29), 4, WL.WATER_MG, m2c.FP64),
                                 ((40, 24, 20), 3, WL.WATER_SG, m2c.MIXED)):
        code, R, L, R_ctx, L_ctx = _case(m2c, n, seed, water, prec)
        assert code == 0
        for v in range(5):
            scale = max(np.abs(R_ctx[v]).max(), 1e-300)
            assert np.abs(R[v] - R_ctx[v]).max() <= 1e-11 * scale
        assert np.abs(L - L_ctx).max() <= 1e-11 * max(np.abs(L_ctx).max(), 1.0)


def test_noalloc_rejects_grids_above_its_maximum():
    """The size check runs on the host before any device work (the array pointers are never
    dereferenced, so this runs without a GPU)."""
    from paper_2508_16387_gb300 import m2c as M
    L = M.lib()
    e0, e1 = M.eos_desc(WL.WATER_SG), M.eos_desc(WL.AIR_PG)
    fake = ctypes.c_void_p(256)
    # 128 x 64 x 33 = 270336 cells > 262144
    code = L.m2c_residual_noalloc(128, 64, 33, 1.0 / 128, (ctypes.c_int * 6)(*(0,) * 6), ctypes.byref(e0),
                                  ctypes.byref(e1), M.FP64, fake, fake, fake, fake, None)
    assert code == M.M2C_EINVAL
    assert b"exceed" in L.m2c_last_error(None)
    assert M.m2c_residual_noalloc_scratch_bytes() < 16 * 2 ** 20


@pytest.mark.parametrize("eos0,eos1,bc,why", [
    ((7, (1.4, 0.0)), WL.AIR_PG, (0,) * 6, "material 0 EOS: unknown EOS type"),
    (WL.WATER_SG, (0, (0.9, 0.0)), (0,) * 6, "material 1 EOS: SG needs gamma > 1"),
    ((1, (1000.0, 1483.0, 0.5, 0.28, 0.0, -float("inf"))), WL.AIR_PG, (0,) * 6,
     "material 0 EOS: MG needs rho0, c0 > 0, s > 1"),
    (WL.WATER_SG, WL.AIR_PG, (0, 0, 9, 9, 0, 0), "unknown boundary condition"),
    (WL.WATER_SG, WL.AIR_PG, (1, 0, 0, 0, 0, 0), "periodic on one side of an axis only"),
    (WL.WATER_SG, WL.AIR_PG, (2, 0, 0, 0, 0, 0), "transmissive and periodic sides only"),
])
def test_noalloc_rejects_bad_eos_and_boundaries_before_any_device_work(eos0, eos1, bc, why):
    """The EOS and boundary rules of m2c_set_eos and m2c_init_grid apply to the allocation-free
    entry point too: a bad EOS type or parameter, or an unknown boundary type, is rejected on the
    host with the reason in m2c_last_error(NULL) (the array pointers are never dereferenced, so
    this runs without a GPU)."""
    from paper_2508_16387_gb300 import m2c as M
    L = M.lib()
    e0, e1 = M.eos_desc(eos0), M.eos_desc(eos1)
    fake = ctypes.c_void_p(256)
    code = L.m2c_residual_noalloc(8, 8, 8, 0.125, (ctypes.c_int * 6)(*bc), ctypes.byref(e0), ctypes.byref(e1),
                                  M.FP64, fake, fake, fake, fake, None)
    assert code == M.M2C_EINVAL
    assert L.m2c_last_error(None).decode().startswith("m2c_residual_noalloc: " + why)
