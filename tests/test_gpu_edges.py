"""Edge cases of the GPU path against the oracle: degenerate and ragged grid
shapes (one-cell axes, tiles cut by the grid edge, periodic axes of two
cells), a bubble cut by the domain boundary, the interface work lists
overflowing, and grids without any axis to move along."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2508_16387_gb300 import workloads as WL

from test_gpu_parity import gpu_start, oracle_start, rel_err  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def m2c():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2508_16387_gb300 import m2c as M
    M.lib()
    return M


@pytest.mark.parametrize("n,bc,two_phase", [
    ((1, 6, 1), (1, 1, 0, 0, 1, 1), True),     # only y moves
    ((40, 1, 1), (0, 0, 1, 1, 1, 1), True),    # 1D along x
    ((3, 1, 7), (0, 0, 0, 0, 1, 1), True),     # thin slab, periodic z
    ((2, 2, 2), (1, 1, 1, 1, 1, 1), False),    # periodic axes of two cells
    ((33, 9, 5), (0, 0, 1, 1, 0, 0), True),    # one cell past a tile in x, ragged y
    ((31, 17, 3), (1, 1, 0, 0, 0, 0), True),   # x narrower than a tile
])
def test_degenerate_and_ragged_shapes(m2c, n, bc, two_phase):
    P, phi = WL.random_state(n, seed=13, two_phase=two_phase)
    if two_phase and not (phi < 0).any():
        phi = phi - np.median(phi)
    s = WL.Setup("edge", n, 1.0 / max(n), (WL.WATER_SG, WL.AIR_PG), bc, phi, np.zeros(phi.shape, np.uint8), {},
                 reinit_every=2, reinit_iters=2)
    g_or, W0 = oracle_start(s, P)
    ref = O.run(g_or, W0, phi, 5)
    g = gpu_start(m2c, s, prims=P)
    g.step(5)
    g.sync()
    assert max(rel_err(g.W.cpu().numpy(), ref.W)) <= 1e-9
    assert np.array_equal(g.phi.cpu().numpy() < 0, ref.phi < 0)


def test_bubble_cut_by_the_boundary(m2c):
    s = WL.shock_bubble(n=32, radius=0.2, centre=(0.55, 0.05, 0.5), steps=40)
    g_or, W0 = oracle_start(s)
    ref = O.run(g_or, W0, s.phi, 40)
    g = gpu_start(m2c, s)
    g.step(40)
    g.sync()
    assert max(rel_err(g.W.cpu().numpy(), ref.W)) <= 1e-9
    assert np.array_equal(g.phi.cpu().numpy() < 0, ref.phi < 0)


def test_interface_list_overflow_is_reported(m2c):
    n = (16, 16, 16)
    x, y, z = np.meshgrid(np.arange(16), np.arange(16), np.arange(16), indexing="ij")
    phi = np.where((x + y + z) % 2 == 0, 0.01, -0.01).transpose(2, 1, 0).copy()  # every face an interface
    P = np.zeros((5,) + phi.shape)
    P[0] = np.where(phi < 0, 1.2, 1000.0)
    P[4] = 1e5
    s = WL.Setup("checker", n, 1.0 / 16, (WL.WATER_SG, WL.AIR_PG), (0,) * 6, phi, np.zeros(phi.shape, np.uint8), {})
    g = gpu_start(m2c, s, prims=P)
    g.step(1)
    code, cell = g.sync_status()
    assert code == 8          # M2C_EOVERFLOW, latched, no fault


def test_grid_without_a_moving_axis_is_rejected(m2c):
    with pytest.raises(m2c.M2CError):
        m2c.Grid((1, 1, 1), 0.1, (0,) * 6, (WL.WATER_SG, WL.AIR_PG))
    g = O.Grid(n=(1, 1, 1), h=0.1, eos=(O.EOS(*WL.WATER_SG), O.EOS(*WL.AIR_PG)))
    with pytest.raises(O.OracleError):
        O.time_step(g, np.ones((5, 1, 1, 1)), np.ones((1, 1, 1)))


@pytest.mark.parametrize("prec,tilings", [
    (0, [(8, 0), (4, 0), (8, 16), (4, 7)]),
    (1, [(8, 0), (16, 0), (4, 8), (16, 32), (8, 5)]),
])
def test_results_do_not_depend_on_the_tiling(m2c, prec, tilings):
    """Every face is computed once, by one formula, whatever the tile that owns it. FP64: the
    state after several steps (reinitialisation included) is bitwise the same for every tile
    shape and z-chunk length, ragged chunks included. Mixed: the compiler may contract FP32
    multiply-adds differently in the code that opens a z-chunk and in the kernel
    instantiated for another tile height, so results agree to FP32 rounding (here within
    1e-5 of each component's scale) rather than bitwise."""
    s = WL.shock_bubble(n=48, radius=0.2, x_shock=0.3, steps=12, water=WL.WATER_MG if prec else WL.WATER_SG)
    ref = None
    for rows, tz in tilings:
        g = gpu_start(m2c, s, prec)
        g.set_tiling(rows, tz)
        g.step(12)
        g.sync()
        out = (g.W.cpu().numpy(), g.phi.cpu().numpy())
        if ref is None:
            ref = out
        elif prec == 0:
            assert np.array_equal(out[0], ref[0]) and np.array_equal(out[1], ref[1]), (rows, tz)
        else:
            assert max(rel_err(out[0], ref[0])) < 1e-5, (rows, tz)
            assert np.abs(out[1] - ref[1]).max() < 1e-6 * s.h * s.n[0], (rows, tz)
    assert (ref[1] < 0).any()
