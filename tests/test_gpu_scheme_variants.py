"""The paper's other scheme choices on the GPU against the oracle's: TVD RK3 and
forward Euler with a constant time step (Sec. 4.3), the MC limiter (App. D,
Eq. theta) and the local Lax-Friedrichs flux (App. C.1), through
m2c_set_options (the general instantiation of the bulk kernel).

Bar: one stage residual <= 1e-11 (normwise); full FP64 runs
<= 1e-9 for the density, the momentum vector and the energy with an identical
sign pattern of phi; the
mixed path <= 1e-4 relative L1 of 4^3-block averages of rho and p.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2508_16387_gb300 import workloads as WL
from tests.metrics import conserved_errors

pytestmark = pytest.mark.gpu

TOL = 1e-9

VARIANTS = {
    "rk3": dict(rk=3),
    "mc": dict(limiter=1, mc_alpha=1.2),
    "llf": dict(flux=1),
    "rk3_mc_llf": dict(rk=3, limiter=1, mc_alpha=1.5, flux=1),
}


@pytest.fixture(scope="module")
def m2c():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2508_16387_gb300 import m2c as M
    M.lib()
    return M


def oracle_grid(s, opts):
    return O.Grid(n=s.n, h=s.h, eos=tuple(O.EOS(*e) for e in s.eos), bc=s.bc, cfl=s.cfl,
                  reinit_every=s.reinit_every, reinit_iters=s.reinit_iters, **opts)


def shocked_prims(s, shock_state):
    if s.shock is None:
        return s.prims()
    amb = s.prims_by_region[s.shock[1]]
    r1, u1, _ = shock_state(s.eos[0], (amb[0], amb[1], amb[4]), s.shock[0])
    return s.prims((r1, u1))


def gpu_grid(M, s, opts, precision=0, prims=None):
    g = M.Grid(s.n, s.h, s.bc, s.eos, precision=precision, cfl=s.cfl, reinit_every=s.reinit_every,
               reinit_iters=s.reinit_iters, options=opts)
    P = prims if prims is not None else shocked_prims(s, M.m2c_shock_state)
    g.set_prims(P, s.phi)
    return g


def oracle_run(s, opts, steps, prims=None):
    g = oracle_grid(s, opts)
    P = prims if prims is not None else shocked_prims(s, lambda e, w, p: O.shock_state(O.EOS(*e), w, p))
    return O.run(g, O.prims_to_cons(g, P, s.phi), s.phi, steps)


# density, momentum vector and energy, normwise (Reading R29)
rel_err = conserved_errors


@pytest.mark.parametrize("name", ["mc", "llf", "rk3_mc_llf"])
@pytest.mark.parametrize("water", [WL.WATER_SG, WL.WATER_MG])
def test_stage_residual_variants_match_oracle(m2c, name, water):
    n = (45, 19, 13)
    P, phi = WL.random_state(n, seed=8, eos=(water, WL.AIR_PG), two_phase=True)
    s = WL.Setup("rand", n, 1.0 / n[0], (water, WL.AIR_PG), (0, 0, 1, 1, 0, 0), phi,
                 np.zeros(phi.shape, np.uint8), {})
    opts = VARIANTS[name]
    g_or = oracle_grid(s, opts)
    R_ref, L_ref, st = O.residual(g_or, O.prims_to_cons(g_or, P, phi), phi)
    g = gpu_grid(m2c, s, opts, prims=P)
    R, L = g.residual()
    R, L = R.cpu().numpy(), L.cpu().numpy()
    assert max(rel_err(R, R_ref)) < 1e-11, rel_err(R, R_ref)
    assert np.abs(L - L_ref).max() <= 1e-11 * max(np.abs(L_ref).max(), 1.0)
    assert st["interface_faces"] > 0


@pytest.mark.parametrize("name", list(VARIANTS))
def test_ragged_bubble_variants_100_steps(m2c, name):
    s = WL.shock_bubble(n=40, radius=0.18, centre=(0.47, 0.52, 0.5), p_shock=8e8, steps=100)
    opts = VARIANTS[name]
    ref = oracle_run(s, opts, 100)
    g = gpu_grid(m2c, s, opts)
    g.step(100)
    t, k = g.sync()
    assert k == 100
    errs = rel_err(g.W.cpu().numpy(), ref.W)
    assert max(errs) <= TOL, errs
    assert np.array_equal(g.phi.cpu().numpy() < 0, ref.phi < 0)
    assert abs(t - ref.t) <= 1e-12 * ref.t


@pytest.mark.parametrize("name", ["rk3", "rk3_mc_llf"])
def test_mg_bubble_variants_60_steps(m2c, name):
    s = WL.shock_bubble(n=36, radius=0.2, water=WL.WATER_MG, steps=60)
    opts = VARIANTS[name]
    ref = oracle_run(s, opts, 60)
    g = gpu_grid(m2c, s, opts)
    g.step(60)
    g.sync()
    assert max(rel_err(g.W.cpu().numpy(), ref.W)) <= TOL
    assert np.array_equal(g.phi.cpu().numpy() < 0, ref.phi < 0)


def test_forward_euler_with_a_constant_time_step(m2c):
    """Forward Euler (Sec. 4.3) on the water-air shock tube with a constant time step a sixth
    of the CFL one: 100 steps, the time advances by exactly 100 dt."""
    s = WL.shock_tube(128, 4, 4, steps=100)
    opts = dict(rk=1, dt_fixed=2.0e-7)
    ref = oracle_run(s, opts, 100)
    g = gpu_grid(m2c, s, opts)
    g.step(100)
    t, k = g.sync()
    assert max(rel_err(g.W.cpu().numpy(), ref.W)) <= TOL
    assert np.array_equal(g.phi.cpu().numpy() < 0, ref.phi < 0)
    assert abs(t - 100 * 2.0e-7) <= 1e-15 and abs(t - ref.t) <= 1e-18
    assert g.stats().interface_faces == ref.stats["interface_faces"]


def test_rk3_with_a_constant_time_step(m2c):
    s = WL.shock_tube(128, 4, 4, steps=150)
    opts = dict(rk=3, dt_fixed=1.0e-6, flux=1)
    ref = oracle_run(s, opts, 150)
    g = gpu_grid(m2c, s, opts)
    g.step(150)
    t, k = g.sync()
    assert max(rel_err(g.W.cpu().numpy(), ref.W)) <= TOL
    assert np.array_equal(g.phi.cpu().numpy() < 0, ref.phi < 0)


@pytest.mark.parametrize("name", ["rk3", "mc", "llf"])
def test_mixed_precision_variants_against_the_oracle(m2c, name):
    s = WL.shock_bubble(n=48, water=WL.WATER_MG, steps=80)
    opts = VARIANTS[name]
    ref = oracle_run(s, opts, 80)
    g = gpu_grid(m2c, s, opts, precision=1)
    g.step(80)
    g.sync()
    g_or = oracle_grid(s, opts)
    P = O.cons_to_prims(g_or, g.W.cpu().numpy(), g.phi.cpu().numpy())
    Pref = O.cons_to_prims(g_or, ref.W, ref.phi)
    for v in (0, 4):
        A = P[v].reshape(12, 4, 12, 4, 12, 4).mean(axis=(1, 3, 5))
        B = Pref[v].reshape(12, 4, 12, 4, 12, 4).mean(axis=(1, 3, 5))
        assert np.abs(A - B).sum() / np.abs(B).sum() <= 1e-4, (name, v)


def test_batch_of_rk3_grids_matches_the_oracle(m2c):
    """Grids with scheme options in one batch (the general kernel over all of them)."""
    params = WL.draw_instances(count=3, seed=5, edges=(16, 24, 20), steps=10)
    setups = [WL.shock_bubble(q.edge, q.radius, q.centre, q.p_shock, steps=q.steps) for q in params]
    opts = [dict(rk=3), dict(rk=3, limiter=1, mc_alpha=1.2), dict(rk=3, flux=1)]
    grids = [gpu_grid(m2c, s, o) for s, o in zip(setups, opts)]
    b = m2c.Batch(grids, (16, 0, 1, 1))  # the general kernel runs 8-row tiles whatever is asked
    b.step(10)
    for s, o, g in zip(setups, opts, grids):
        g.sync()
        ref = oracle_run(s, o, 10)
        assert max(rel_err(g.W.cpu().numpy(), ref.W)) <= TOL
        assert np.array_equal(g.phi.cpu().numpy() < 0, ref.phi < 0)


def test_option_errors(m2c):
    s = WL.shock_bubble(n=16, steps=1)
    g = gpu_grid(m2c, s, None)
    for bad in (dict(rk=4), dict(limiter=2), dict(flux=3), dict(limiter=1, mc_alpha=2.5), dict(dt_fixed=-1.0)):
        with pytest.raises(m2c.M2CError) as e:
            g.set_options(**bad)
        assert e.value.code == 1
    # TVD RK3 needs the larger workspace (the Grid above was sized for RK2)
    with pytest.raises(m2c.M2CError) as e:
        g.set_options(rk=3)
    assert e.value.code == 2
    g.set_options(limiter=1)
    with pytest.raises(m2c.M2CError):
        g.set_tiling(4)
