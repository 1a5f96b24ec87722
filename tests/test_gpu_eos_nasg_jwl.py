"""The Noble-Abel stiffened gas (Sec. 3.3, Eq. NASG_EOS) and the Jones-Wilkins-Lee
EOS (App. B.2, Eq. JWL_EOS; Readings R35, R36) on the GPU against the oracle: the
exact two-material Riemann solve of the FIVER flux (batch <= 1e-10 with equal
iteration counts), the stage residual (<= 1e-11), FP64 runs (<= 1e-9 for the
density, the momentum vector and the energy, identical sign of phi), the mixed
path (<= 1e-4 relative L1 of rho and p) and the post-shock state."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2508_16387_gb300 import workloads as WL
from tests.metrics import conserved_errors as rel_err

pytestmark = pytest.mark.gpu

TOL = 1e-9
LIQ, JWL, AIR, WATER, WATER_MG = WL.LIQUID_NASG, WL.PRODUCTS_JWL, WL.AIR_PG, WL.WATER_SG, WL.WATER_MG
GAS_NASG = (WL.EOS_NASG, (1.4, 0.0, 1.0e-3, 0.0))


@pytest.fixture(scope="module")
def m2c():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2508_16387_gb300 import m2c as M
    M.lib()
    return M


def states(rng, kind, n):
    if kind == "air":
        return np.stack([rng.uniform(0.5, 5.0, n), rng.uniform(-300, 300, n), rng.uniform(5e4, 5e6, n)])
    if kind == "gas":
        return np.stack([rng.uniform(0.5, 50.0, n), rng.uniform(-300, 300, n), rng.uniform(5e4, 5e7, n)])
    if kind == "jwl":
        return np.stack([rng.uniform(1000, 1700, n), rng.uniform(-300, 300, n), rng.uniform(1e9, 3e10, n)])
    return np.stack([rng.uniform(950, 1250, n), rng.uniform(-300, 300, n), rng.uniform(1e5, 2e9, n)])


EOS = {"liq": LIQ, "gas": GAS_NASG, "jwl": JWL, "air": AIR, "water": WATER, "mg": WATER_MG}


@pytest.mark.parametrize("pair", ["liq_air", "liq_gas", "jwl_air", "jwl_water", "mg_jwl", "air_jwl", "liq_liq"])
def test_riemann_batch_matches_oracle(m2c, pair):
    import torch
    rng = np.random.default_rng(21)
    n = 2048
    a, b = pair.split("_")
    L, R = states(rng, a if a != "mg" else "water", n), states(rng, b if b != "mg" else "water", n)
    ref, rit, rst = O.riemann_batch(O.EOS(*EOS[a]), L, O.EOS(*EOS[b]), R)
    for mixed in (False, True):  # the FP32 start leaves NASG and JWL problems to the FP64 iteration
        out, it, st = m2c.m2c_solve_riemann(EOS[a], torch.from_numpy(L).cuda(), EOS[b], torch.from_numpy(R).cuda(),
                                            mixed=mixed)
        out, it, st = out.cpu().numpy(), it.cpu().numpy(), st.cpu().numpy()
        assert np.array_equal(st, rst)
        ok = rst == 0
        assert ok.mean() > 0.9
        for v in range(4):
            scale = np.maximum(np.abs(ref[v][ok]), 1e-3 if v == 1 else 1e-300)
            assert np.max(np.abs(out[v][ok] - ref[v][ok]) / scale) < 1e-10, (mixed, v)
        if not mixed:
            assert np.array_equal(it[ok], rit[ok])


@pytest.mark.parametrize("eos", [LIQ, JWL])
def test_shock_state_matches_oracle(m2c, eos):
    w = (1000.0, 0.0, 1e5) if eos is LIQ else (1600.0, 0.0, 1e9)
    p1 = 2e9 if eos is LIQ else 2e10
    g = m2c.m2c_shock_state(eos, w, p1)
    r = O.shock_state(O.EOS(*eos), w, p1)
    assert np.allclose(g, r, rtol=1e-12)


def _setup(n, mat0, base0, seed):
    P, phi = WL.random_state(n, seed=seed, eos=(mat0, AIR), two_phase=True, base={0: base0, 1: (1.2, 1e5)})
    s = WL.Setup("rand", n, 1.0 / n[0], (mat0, AIR), (0, 0, 1, 1, 0, 0), phi, np.zeros(phi.shape, np.uint8), {})
    return s, P, phi


@pytest.mark.parametrize("mat", ["liq", "jwl"])
def test_stage_residual_matches_oracle(m2c, mat):
    n = (41, 19, 15)
    s, P, phi = _setup(n, EOS[mat], (1000.0, 1e8) if mat == "liq" else (1400.0, 5e9), seed=17)
    g_or = O.Grid(n=n, h=s.h, eos=(O.EOS(*EOS[mat]), O.EOS(*AIR)), bc=s.bc)
    R_ref, L_ref, st = O.residual(g_or, O.prims_to_cons(g_or, P, phi), phi)
    for prec, tol in ((0, 1e-11),):
        g = m2c.Grid(n, s.h, s.bc, (EOS[mat], AIR), precision=prec)
        g.set_prims(P, phi)
        R, L = g.residual()
        R, L = R.cpu().numpy(), L.cpu().numpy()
        assert max(rel_err(R, R_ref)) < tol
        assert np.abs(L - L_ref).max() <= tol * max(np.abs(L_ref).max(), 1.0)
    assert st["interface_faces"] > 0


def _bubble_in(mat, n):
    """A bubble of air in a liquid (NASG) at 1e5 Pa hit by a planar 1.5e9 Pa shock, or a
    sphere of detonation products (JWL, 1600 kg/m^3, 2e10 Pa) in air."""
    h = 1.0 / n
    x, y, z = WL.cell_centres((n, n, n), h)
    if mat == "liq":
        phi = np.sqrt((x - 0.55) ** 2 + (y - 0.5) ** 2 + (z - 0.5) ** 2) - 0.2
        P = np.zeros((5,) + phi.shape)
        P[0] = np.where(phi < 0, 1.2, 1000.0)
        P[4] = 1e5
        r1, u1, _ = O.shock_state(O.EOS(*LIQ), (1000.0, 0.0, 1e5), 1.5e9)
        sh = (x < 0.25) & (phi >= 0)
        P[0][sh], P[1][sh], P[4][sh] = r1, u1, 1.5e9
        return (LIQ, AIR), P, phi
    # products where phi < 0 (material 1), air outside
    phi = np.sqrt((x - 0.5) ** 2 + (y - 0.5) ** 2 + (z - 0.5) ** 2) - 0.15
    P = np.zeros((5,) + phi.shape)
    P[0] = np.where(phi < 0, 1600.0, 1.2)
    P[4] = np.where(phi < 0, 2e10, 1e5)
    return (AIR, JWL), P, phi


# the JWL rarefaction integrates hundreds of RK4 substeps per unit of ln p in every evaluation,
# so its run is kept small for the oracle's sake
@pytest.mark.parametrize("mat,n,steps", [("liq", 32, 80), ("jwl", 20, 16)])
def test_two_material_runs_match_oracle(m2c, mat, n, steps):
    eos, P, phi = _bubble_in(mat, n)
    g_or = O.Grid(n=(n, n, n), h=1.0 / n, eos=tuple(O.EOS(*e) for e in eos), bc=(0,) * 6)
    ref = O.run(g_or, O.prims_to_cons(g_or, P, phi), phi, steps)
    g = m2c.Grid((n, n, n), 1.0 / n, (0,) * 6, eos)
    g.set_prims(P, phi)
    g.step(steps)
    t, k = g.sync()
    assert max(rel_err(g.W.cpu().numpy(), ref.W)) <= TOL
    assert np.array_equal(g.phi.cpu().numpy() < 0, ref.phi < 0)
    assert abs(t - ref.t) <= 1e-12 * ref.t
    # mixed precision against the same oracle run
    gm = m2c.Grid((n, n, n), 1.0 / n, (0,) * 6, eos, precision=1)
    gm.set_prims(P, phi)
    gm.step(steps)
    gm.sync()
    Pg = O.cons_to_prims(g_or, gm.W.cpu().numpy(), gm.phi.cpu().numpy())
    Pr = O.cons_to_prims(g_or, ref.W, ref.phi)
    for v in (0, 4):
        k = n // 4
        A = Pg[v].reshape(k, 4, k, 4, k, 4).mean(axis=(1, 3, 5))
        B = Pr[v].reshape(k, 4, k, 4, k, 4).mean(axis=(1, 3, 5))
        assert np.abs(A - B).sum() / np.abs(B).sum() <= 1e-4, (mat, v)


def test_eos_parameter_errors(m2c):
    g = m2c.Grid((8, 8, 8), 0.1, (0,) * 6, (WATER, AIR))
    L = m2c.lib()
    import ctypes
    for t, prm in ((2, (0.9, 0.0, 0.0, 0.0)), (2, (1.4, 0.0, -1e-3, 0.0)), (2, (1.4, 0.0, 0.0)),
                   (3, (0.0, 1e11, 1e9, 4.5, 1.0, 1600.0)), (3, (0.3, 1e11, 1e9, 4.5, 1.0, -1.0))):
        arr = (ctypes.c_double * 6)(*(list(prm) + [0.0] * (6 - len(prm))))
        assert L.m2c_set_eos(g.ctx, 0, t, arr, len(prm)) == 1
