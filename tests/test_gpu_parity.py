"""GPU FP64 path against the CPU oracle, element by element, through the C-ABI.

Both sides start from the same seeded primitive fields and build their own
conserved state (each with its own EOS and its own post-shock state).
Tolerance: max_cells |W_gpu - W_oracle| / max_cells |W_oracle| <= 1e-9 for the
density, the momentum vector (Euclidean norm) and the energy after the stated
steps, and an identical sign pattern of phi (the material map).
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2508_16387_gb300 import workloads as WL
from tests.metrics import conserved_errors

pytestmark = pytest.mark.gpu

TOL = 1e-9


@pytest.fixture(scope="module")
def m2c():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2508_16387_gb300 import m2c as M
    M.lib()
    return M


def oracle_grid(s):
    return O.Grid(n=s.n, h=s.h, eos=tuple(O.EOS(*e) for e in s.eos), bc=s.bc, cfl=s.cfl,
                  reinit_every=s.reinit_every, reinit_iters=s.reinit_iters)


def oracle_start(s, prims=None):
    g = oracle_grid(s)
    if prims is None:
        shocked = None
        if s.shock is not None:
            amb = s.prims_by_region[s.shock[1]]
            r1, u1, _ = O.shock_state(O.EOS(*s.eos[0]), (amb[0], amb[1], amb[4]), s.shock[0])
            shocked = (r1, u1)
        prims = s.prims(shocked)
    return g, O.prims_to_cons(g, prims, s.phi)


def gpu_start(M, s, precision=0, prims=None):
    g = M.Grid(s.n, s.h, s.bc, s.eos, precision=precision, cfl=s.cfl, reinit_every=s.reinit_every,
               reinit_iters=s.reinit_iters)
    if prims is None:
        shocked = None
        if s.shock is not None:
            amb = s.prims_by_region[s.shock[1]]
            r1, u1, _ = M.m2c_shock_state(s.eos[0], (amb[0], amb[1], amb[4]), s.shock[0])
            shocked = (r1, u1)
        prims = s.prims(shocked)
    g.set_prims(prims, s.phi)
    return g


def prim_err(a, b):
    return [float(np.abs(a[v] - b[v]).max() / max(np.abs(b[v]).max(), 1e-300)) for v in range(a.shape[0])]


# conserved states and residuals: density, momentum vector and energy, normwise (Reading R29)
rel_err = conserved_errors


# --------------------------------------------------------------------------- Riemann solver

@pytest.mark.parametrize("pair", ["sg_sg", "sg_pg", "mg_pg", "mg_mg"])
def test_riemann_batch_matches_oracle(m2c, pair):
    import torch
    rng = np.random.default_rng(11)
    n = 4096
    eos = {"sg": WL.WATER_SG, "pg": WL.AIR_PG, "mg": WL.WATER_MG}
    a, b = pair.split("_")
    eL, eR = eos[a], eos[b]

    def states(kind):
        if kind == "pg":
            return np.stack([rng.uniform(0.5, 5.0, n), rng.uniform(-300, 300, n), rng.uniform(5e4, 5e6, n)])
        return np.stack([rng.uniform(950, 1250, n), rng.uniform(-300, 300, n), rng.uniform(1e5, 2e9, n)])
    L, R = states(a), states(b)
    ref, rit, rst = O.riemann_batch(O.EOS(*eL), L, O.EOS(*eR), R)
    out, it, st = m2c.m2c_solve_riemann(eL, torch.from_numpy(L).cuda(), eR, torch.from_numpy(R).cuda())
    out, it, st = out.cpu().numpy(), it.cpu().numpy(), st.cpu().numpy()
    assert np.array_equal(st, rst)
    ok = rst == 0
    assert ok.mean() > 0.9
    for v in range(4):
        scale = np.maximum(np.abs(ref[v][ok]), 1e-3 if v == 1 else 1e-300)
        assert np.max(np.abs(out[v][ok] - ref[v][ok]) / scale) < 1e-10, v
    assert np.array_equal(it[ok], rit[ok])


def _sound_speed(eos, rho, p):
    try:
        return float(np.sqrt(O.sound_speed2(O.EOS(*eos), rho, p)))
    except O.OracleError:
        return float("nan")


@pytest.mark.parametrize("pair", ["sg_pg", "mg_pg", "pg_mg", "sg_sg", "mg_mg"])
def test_riemann_mixed_batch_matches_oracle(m2c, pair):
    """The mixed path's Riemann solve (FP32 Newton, then FP64 Newton steps) against the
    FP64 oracle on wide random states and on near-equilibrium states like those at a
    bubble surface at rest, down to rounding-level differences (where a shock curve's
    slope is not finite in FP64 and the FP64 iteration takes over)."""
    import torch
    rng = np.random.default_rng(12)
    n = 4096
    eos = {"sg": WL.WATER_SG, "pg": WL.AIR_PG, "mg": WL.WATER_MG}
    a, b = pair.split("_")
    eL, eR = eos[a], eos[b]

    def states(kind, quiet):
        if quiet is not None:  # 1e5 Pa at rest with relative perturbations of size quiet
            rho = 1.2 if kind == "pg" else 1000.0
            return np.stack([rho * (1 + quiet * rng.standard_normal(n)), 10 * quiet * rng.standard_normal(n),
                             1e5 * (1 + quiet * rng.standard_normal(n))])
        if kind == "pg":
            return np.stack([rng.uniform(0.5, 5.0, n), rng.uniform(-300, 300, n), rng.uniform(5e4, 5e6, n)])
        return np.stack([rng.uniform(950, 1250, n), rng.uniform(-300, 300, n), rng.uniform(1e5, 2e9, n)])
    for quiet in (None, 1e-4, 1e-8, 1e-12, 0.0):
        L, R = states(a, quiet), states(b, quiet)
        ref, _, rst = O.riemann_batch(O.EOS(*eL), L, O.EOS(*eR), R)
        out, it, st = m2c.m2c_solve_riemann(eL, torch.from_numpy(L).cuda(), eR, torch.from_numpy(R).cuda(),
                                            mixed=True)
        out, st = out.cpu().numpy(), st.cpu().numpy()
        assert np.array_equal(st, rst)
        ok = rst == 0
        assert ok.mean() > 0.9
        assert np.isfinite(out[:, ok]).all()
        # both iterations run on the same wave curves (the RK4 substep count of an MG
        # rarefaction is fixed per problem before the iteration) and stop within rounding of
        # the same root: p* and rho* to 1e-10 relative, u* to 1e-11 of the problem's velocity
        # scale max(|u_L|, |u_R|, c_L, c_R)
        cL = np.array([_sound_speed(eL, L[0, i], L[2, i]) for i in range(n)])
        cR = np.array([_sound_speed(eR, R[0, i], R[2, i]) for i in range(n)])
        uscale = np.maximum.reduce([np.abs(L[1]), np.abs(R[1]), cL, cR])[ok]
        assert np.max(np.abs(out[0][ok] - ref[0][ok]) / np.abs(ref[0][ok])) < 1e-10, quiet
        assert np.max(np.abs(out[1][ok] - ref[1][ok]) / uscale) < 1e-11, quiet
        for v in (2, 3):
            assert np.max(np.abs(out[v][ok] - ref[v][ok]) / ref[v][ok]) < 1e-10, (quiet, v)


def test_riemann_host_arrays_and_shock_state(m2c):
    L = np.array([[1000.0], [0.0], [1e9]])
    R = np.array([[1.0], [0.0], [1e5]])
    code, out, it, st = m2c.m2c_solve_riemann_host(WL.WATER_SG, L, WL.AIR_PG, R)
    assert code == 0
    ref, _ = O.riemann(O.EOS(*WL.WATER_SG), L[:, 0], O.EOS(*WL.AIR_PG), R[:, 0])
    assert np.allclose(out[:, 0], ref, rtol=1e-12)
    for eos in (WL.WATER_SG, WL.WATER_MG):
        g = m2c.m2c_shock_state(eos, (1000.0, 0.0, 1e5), 1e9)
        r = O.shock_state(O.EOS(*eos), (1000.0, 0.0, 1e5), 1e9)
        assert np.allclose(g, r, rtol=1e-12)
    # vacuum is reported, not solved
    code, out, it, st = m2c.m2c_solve_riemann_host(WL.AIR_PG, np.array([[1.0], [-2e4], [1e5]]), WL.AIR_PG,
                                                   np.array([[1.0], [2e4], [1e5]]))
    assert code == 6 and st[0] == 6


@pytest.mark.parametrize("mixed", [False, True])
def test_riemann_near_vacuum_matches_oracle(m2c, mixed):
    """Expansion problems on both sides of the vacuum threshold (air | air: u_R - u_L =
    4c/(gamma - 1) = 3741.7 m/s; water | air with a stiffened and a Mie-Grueneisen water, near
    2c_air/(gamma - 1) = 1708 m/s): the GPU
    solver tests F(p_low) >= 0 only when its Newton iteration has not converged (a root above
    p_low rules a vacuum out), the oracle before it; the status agrees everywhere, and so does
    the solution where there is one."""
    cases = []
    for du in (1000.0, 3000.0, 3700.0, 3780.0, 3900.0, 6000.0):
        cases.append((WL.AIR_PG, (1.0, -0.5 * du, 1e5), WL.AIR_PG, (1.0, 0.5 * du, 1e5)))
    for water in (WL.WATER_SG, WL.WATER_MG):
        for du in (100.0, 1000.0, 1650.0, 1750.0, 2000.0, 4500.0):
            cases.append((water, (1000.0, -0.5 * du, 1e5), WL.AIR_PG, (1.2, 0.5 * du, 1e5)))
    for eL, wL, eR, wR in cases:
        code, out, it, st = m2c.m2c_solve_riemann_host(eL, np.array(wL).reshape(3, 1), eR, np.array(wR).reshape(3, 1),
                                                       mixed=mixed)
        ref_st = O.riemann_status(O.EOS(*eL), wL, O.EOS(*eR), wR)
        assert st[0] == ref_st, (eL, wL, eR, wR, st[0], ref_st)
        if ref_st == 0:
            ref, _ = O.riemann(O.EOS(*eL), wL, O.EOS(*eR), wR)
            assert abs(out[0, 0] - ref[0]) <= 1e-9 * abs(ref[0]) + 1e-12 * wL[2], (wL, wR, out[:, 0], ref)
            assert abs(out[1, 0] - ref[1]) <= 1e-9 * max(abs(wL[1]), abs(wR[1]))
            assert np.allclose(out[2:, 0], ref[2:], rtol=1e-8)


@pytest.mark.parametrize("water", [WL.WATER_SG, WL.WATER_MG])
def test_state_to_prims_matches_oracle(m2c, water):
    """m2c_state_to_prims against the oracle's conversion of the same conserved state, and the
    round trip from primitive fields, on a random two-phase state."""
    n = (29, 17, 11)
    P, phi = WL.random_state(n, seed=5, eos=(water, WL.AIR_PG), two_phase=True)
    s = WL.Setup("rand", n, 1.0 / n[0], (water, WL.AIR_PG), (0, 0, 1, 1, 0, 0), phi,
                 np.zeros(phi.shape, np.uint8), {})
    g = gpu_start(m2c, s, prims=P)
    G = g.prims().cpu().numpy()
    g.sync()
    ref = O.cons_to_prims(oracle_grid(s), g.W.cpu().numpy(), phi)
    assert max(prim_err(G, ref)) < 1e-13
    assert max(prim_err(G, P)) < 1e-11


# --------------------------------------------------------------------------- one stage residual

@pytest.mark.parametrize("n,two_phase,water", [((70, 19, 13), True, WL.WATER_SG), ((45, 33, 9), True, WL.WATER_MG),
                                               ((37, 11, 17), False, WL.WATER_SG)])
def test_stage_residual_matches_oracle(m2c, n, two_phase, water):
    P, phi = WL.random_state(n, seed=7, eos=(water, WL.AIR_PG), two_phase=two_phase)
    s = WL.Setup("rand", n, 1.0 / n[0], (water, WL.AIR_PG), (0, 0, 1, 1, 0, 0), phi,
                 np.zeros(phi.shape, np.uint8), {})
    g_or, W0 = oracle_start(s, P)
    R_ref, L_ref, st = O.residual(g_or, W0, phi)
    g = gpu_start(m2c, s, prims=P)
    R, L = g.residual()
    R, L = R.cpu().numpy(), L.cpu().numpy()
    assert max(rel_err(R, R_ref)) < 1e-11
    assert np.abs(L - L_ref).max() <= 1e-11 * max(np.abs(L_ref).max(), 1.0)
    if two_phase:
        assert st["interface_faces"] > 0


# --------------------------------------------------------------------------- full steps

def _run_both(m2c, s, steps, precision=0):
    g_or, W0 = oracle_start(s)
    ref = O.run(g_or, W0, s.phi, steps)
    g = gpu_start(m2c, s, precision)
    g.step(steps)
    t, k = g.sync()
    assert k == steps
    return ref, g.W.cpu().numpy(), g.phi.cpu().numpy(), t, g


def test_shock_tube_200_steps(m2c):
    s = WL.shock_tube(128, 4, 4, steps=200)
    ref, W, phi, t, g = _run_both(m2c, s, 200)
    errs = rel_err(W, ref.W)
    assert max(errs) <= TOL, errs
    assert np.array_equal(phi < 0, ref.phi < 0)
    assert abs(t - ref.t) <= 1e-12 * ref.t
    assert g.stats().interface_faces == ref.stats["interface_faces"]


def test_ragged_bubble_100_steps(m2c):
    s = WL.shock_bubble(n=40, radius=0.18, centre=(0.47, 0.52, 0.5), p_shock=8e8, steps=100)
    ref, W, phi, t, g = _run_both(m2c, s, 100)
    errs = rel_err(W, ref.W)
    assert max(errs) <= TOL, errs
    assert np.array_equal(phi < 0, ref.phi < 0)
    assert ref.stats["flipped"] > 0


def test_mg_bubble_30_steps(m2c):
    s = WL.shock_bubble(n=36, radius=0.2, water=WL.WATER_MG, steps=30)
    ref, W, phi, t, g = _run_both(m2c, s, 30)
    assert max(rel_err(W, ref.W)) <= TOL
    assert np.array_equal(phi < 0, ref.phi < 0)


@pytest.mark.slow
def test_shock_bubble_128_cubed_100_steps(m2c):
    """The 128^3 shock-bubble workload (stiffened-gas water, 1e9 Pa shock), 100 steps."""
    s = WL.shock_bubble(n=128, steps=100)
    ref, W, phi, t, g = _run_both(m2c, s, 100)
    errs = rel_err(W, ref.W)
    assert max(errs) <= TOL, errs
    assert np.array_equal(phi < 0, ref.phi < 0)


@pytest.mark.slow
def test_mg_shock_bubble_256_cubed_one_step(m2c):
    """The 256^3 Mie-Grueneisen shock-bubble workload, FP64, one full step compared cell by cell."""
    s = WL.shock_bubble(n=256, water=WL.WATER_MG, steps=1)
    ref, W, phi, t, g = _run_both(m2c, s, 1)
    assert max(rel_err(W, ref.W)) <= TOL
    assert np.array_equal(phi < 0, ref.phi < 0)


def test_single_material_periodic_conserves(m2c):
    n = (64, 48, 40)
    P, phi = WL.random_state(n, seed=5, two_phase=False)
    s = WL.Setup("per", n, 1.0 / 64, (WL.WATER_SG, WL.AIR_PG), (1,) * 6, phi, np.zeros(phi.shape, np.uint8), {})
    g = gpu_start(m2c, s, prims=P)
    W0 = g.W.cpu().numpy().copy()
    g.step(30)
    g.sync()
    W = g.W.cpu().numpy()
    for v in range(5):
        assert abs(W[v].sum() - W0[v].sum()) <= 1e-13 * np.abs(W0[v]).sum()


@pytest.mark.parametrize("prec", [0, 1])
def test_checkpoint_restart_matches_the_uninterrupted_run(m2c, prec):
    """A run restarted from its (W, phi, t, step) at step 10 against the uninterrupted run at step
    20: the same time and material map, and the state to rounding. Not bit for bit: the FIVER
    Newton iteration of the uninterrupted run starts from each face's star pressure of the
    previous solve, which (W, phi) does not carry (the restart starts from the PVRS estimate); both
    stop at the same root within the iteration's tolerance."""
    s = WL.shock_bubble(n=32, radius=0.2, steps=20, water=WL.WATER_MG if prec else WL.WATER_SG)
    g = gpu_start(m2c, s, prec)
    g.step(20)
    t_full, _ = g.sync()
    W_full = g.W.cpu().numpy()
    g2 = gpu_start(m2c, s, prec)
    g2.step(10)
    t, k = g2.sync()
    Wm, pm = g2.W.cpu().numpy(), g2.phi.cpu().numpy()
    g3 = m2c.Grid(s.n, s.h, s.bc, s.eos, precision=prec)
    g3.set_state(Wm, pm, t=t, step=k)
    g3.step(10)
    t3, k3 = g3.sync()
    assert k3 == 20 and abs(t3 - t_full) <= 1e-13 * t_full
    assert max(rel_err(g3.W.cpu().numpy(), W_full)) <= 1e-12
    assert np.array_equal(g3.phi.cpu().numpy() < 0, g.phi.cpu().numpy() < 0)


def test_nonphysical_state_is_reported(m2c):
    s = WL.shock_bubble(n=24, radius=0.2, steps=2)
    g = gpu_start(m2c, s)
    W = g.W.cpu().numpy()
    W[0, 5, 6, 7] = -1.0
    g.set_state(W, s.phi)
    g.step(1)
    code, cell = g.sync_status()
    assert code == 5
    assert cell == (5 * 24 + 6) * 24 + 7


def _block_l1(a, b, k=4):
    nz, ny, nx = a.shape
    A = a.reshape(nz // k, k, ny // k, k, nx // k, k).mean(axis=(1, 3, 5))
    B = b.reshape(nz // k, k, ny // k, k, nx // k, k).mean(axis=(1, 3, 5))
    return float(np.abs(A - B).sum() / np.abs(B).sum())


@pytest.mark.parametrize("fp32_start", [False, True])
def test_mixed_precision_l1_error_against_fp64(m2c, fp32_start):
    """Mixed precision (FP32 reconstruction and HLLC, FP64 accumulation and Riemann solver; with
    fp32_start the Riemann iteration starts on FP32 curves) on the MG shock-bubble setup at 64^3
    after the shock has reached the bubble: relative L1 error of 4^3-block averages of density
    and pressure against the FP64 path <= 1e-4."""
    s = WL.shock_bubble(n=64, water=WL.WATER_MG, steps=100)
    out = {}
    for prec in (0, 1):
        g = gpu_start(m2c, s, prec)
        if fp32_start:
            if prec == 0:  # an option of mixed grids only
                with pytest.raises(m2c.M2CError):
                    g.set_riemann_start(True)
            else:
                g.set_riemann_start(True)
        g.step(100)
        g.sync()
        W = g.W.cpu().numpy()
        phi = g.phi.cpu().numpy()
        P = O.cons_to_prims(oracle_grid(s), W, phi)
        out[prec] = (P, phi)
    P64, P32 = out[0][0], out[1][0]
    e_rho = _block_l1(P32[0], P64[0])
    e_p = _block_l1(P32[4], P64[4])
    assert e_rho <= 1e-4 and e_p <= 1e-4, (e_rho, e_p)
    assert (out[0][1] < 0).sum() > 0


def test_isolated_flip_matches_oracle(m2c):
    from tests.test_oracle_pins import _undershoot_setup
    s, P = _undershoot_setup()
    g_or, W0 = oracle_start(s, P)
    ref = O.run(g_or, W0, s.phi, 1)
    g = gpu_start(m2c, s, prims=P)
    g.step(1)
    g.sync()
    assert np.array_equal(g.phi.cpu().numpy() < 0, ref.phi < 0)
    assert np.abs(g.phi.cpu().numpy() - ref.phi).max() <= 1e-12
    assert max(rel_err(g.W.cpu().numpy(), ref.W)) <= TOL
