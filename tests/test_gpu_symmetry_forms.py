"""Mirror (symmetry) boundaries and the spherical and cylindrical forms of Sec. 3.4
(Eqs. euler1d_spherical and Euler_cylindrical, Reading R37) on the GPU against the
oracle: residuals <= 1e-11, FP64 runs <= 1e-9 for the density, the momentum
vector and the energy with an identical sign pattern of phi, the mixed path
<= 1e-4 relative L1 of rho and p. The GPU half domain with a mirror side also
reproduces the GPU full domain of a mirror-symmetric problem."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2508_16387_gb300 import workloads as WL
from tests.metrics import conserved_errors as rel_err

pytestmark = pytest.mark.gpu

TOL = 1e-9
S = 2  # BC_SYMMETRY
AIR, WATER = WL.AIR_PG, WL.WATER_SG


@pytest.fixture(scope="module")
def m2c():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2508_16387_gb300 import m2c as M
    M.lib()
    return M


def both(M, n, h, bc, eos, P, phi, steps, opts=None, precision=0, reinit=(10, 5)):
    opts = opts or {}
    g_or = O.Grid(n=n, h=h, eos=tuple(O.EOS(*e) for e in eos), bc=bc, reinit_every=reinit[0],
                  reinit_iters=reinit[1], **opts)
    ref = O.run(g_or, O.prims_to_cons(g_or, P, phi), phi, steps)
    g = M.Grid(n, h, bc, eos, precision=precision, reinit_every=reinit[0], reinit_iters=reinit[1],
               options=opts or None)
    g.set_prims(P, phi)
    g.step(steps)
    t, k = g.sync()
    assert k == steps
    return g_or, ref, g, t


def bubble_in_water(r, R=0.25, p_water=5e8):
    """Air bubble of radius R at r = 0 in compressed water (phi = r - R, air inside)."""
    phi = r - R
    P = np.zeros((5,) + r.shape)
    P[0] = np.where(phi < 0, 1.2, 1000.0)
    P[4] = np.where(phi < 0, 1e5, p_water)
    return P, phi


def test_spherical_bubble_collapse_1d(m2c):
    """The free-field bubble collapse of Sec. 5 in its 1D spherical form (mirror at r = 0): the
    FIVER flux on the bubble wall, the geometric source in the bulk and interface cells."""
    nr = 256
    h = 1.0 / nr
    r = (np.arange(nr) + 0.5) * h
    P, phi = bubble_in_water(r[None, None, :])
    opts = dict(geom=O.GEOM_SPHERICAL, x0=0.0)
    g_or, ref, g, t = both(m2c, (nr, 1, 1), h, (S, 0, 0, 0, 0, 0), (WATER, AIR), P, phi, 300, opts)
    assert max(rel_err(g.W.cpu().numpy(), ref.W)) <= TOL
    assert np.array_equal(g.phi.cpu().numpy() < 0, ref.phi < 0)
    assert abs(t - ref.t) <= 1e-12 * ref.t
    assert ref.stats["flipped"] > 0  # cells changed material over the run


def test_cylindrical_shock_tube(m2c):
    """An air sphere at high pressure in the (r, z) half plane of the cylindrical form, mirror
    sides at r = 0 and z = 0."""
    m = 48
    h = 0.5 / m
    c = (np.arange(m) + 0.5) * h
    z, x = np.meshgrid(c, c, indexing="ij")
    rs = np.sqrt(x * x + z * z)[:, None, :]
    P = np.zeros((5,) + rs.shape)
    P[0] = np.where(rs < 0.2, 1.0, 0.125)
    P[4] = np.where(rs < 0.2, 10.0, 1.0)
    phi = np.ones(rs.shape)
    opts = dict(geom=O.GEOM_CYLINDRICAL, x0=0.0)
    g_or, ref, g, t = both(m2c, (m, 1, m), h, (S, 0, 0, 0, S, 0), (AIR, AIR), P, phi, 120, opts)
    assert max(rel_err(g.W.cpu().numpy(), ref.W)) <= TOL


def test_cylindrical_form_offset_from_the_axis_with_rk3(m2c):
    """An annulus (x0 > 0, transmissive inner side) with TVD RK3 and the MC limiter."""
    m = 40
    h = 0.5 / m
    c = (np.arange(m) + 0.5) * h
    z, x = np.meshgrid(c, c, indexing="ij")
    rr = 0.3 + x
    phi = (np.sqrt((rr - 0.55) ** 2 + (z - 0.25) ** 2) - 0.12)[:, None, :]
    P = np.zeros((5,) + phi.shape)
    P[0] = np.where(phi < 0, 1.2, 1000.0)
    P[1] = np.where(phi < 0, 0.0, 30.0)
    P[4] = np.where(phi < 0, 1e5, 2e8)
    opts = dict(geom=O.GEOM_CYLINDRICAL, x0=0.3, rk=3, limiter=1, mc_alpha=1.3)
    g_or, ref, g, t = both(m2c, (m, 1, m), h, (0, 0, 0, 0, S, 0), (WATER, AIR), P, phi, 60, opts)
    assert max(rel_err(g.W.cpu().numpy(), ref.W)) <= TOL
    assert np.array_equal(g.phi.cpu().numpy() < 0, ref.phi < 0)


def test_octant_shock_bubble_with_three_mirror_sides(m2c):
    """The 3D shock-bubble problem on an octant: the bubble centred on the corner where three
    mirror planes meet, the shock arriving along x; the reinitialisation and the phase update
    read across the mirror planes."""
    n = 40
    h = 0.5 / n
    c = (np.arange(n) + 0.5) * h
    z, y, x = np.meshgrid(c, c, c, indexing="ij")
    phi = np.sqrt(x * x + y * y + z * z) - 0.2
    P = np.zeros((5,) + phi.shape)
    P[0] = np.where(phi < 0, 1.2, 1000.0)
    P[4] = np.where(phi < 0, 1e5, 1e5)
    shocked = (x > 0.38) & (phi >= 0)
    r1, u1, _ = O.shock_state(O.EOS(*WATER), (1000.0, 0.0, 1e5), 1e9)
    P[0][shocked] = r1
    P[1][shocked] = -u1
    P[4][shocked] = 1e9
    g_or, ref, g, t = both(m2c, (n, n, n), h, (S, 0, S, 0, S, 0), (WATER, AIR), P, phi, 80,
                           reinit=(4, 3))
    assert max(rel_err(g.W.cpu().numpy(), ref.W)) <= TOL
    assert np.array_equal(g.phi.cpu().numpy() < 0, ref.phi < 0)
    assert ref.stats["interface_faces"] > 0


def test_mirror_half_domain_equals_the_full_domain(m2c):
    """The half domain x > 1/2 with a mirror side at x = 1/2 (GPU) against the right half of the
    mirror-symmetric full domain (GPU), and against the oracle's half domain."""
    n = 32
    h = 1.0 / n
    c = (np.arange(n) + 0.5) * h
    z, y, x = np.meshgrid(c, c, c, indexing="ij")
    phi = np.sqrt((x - 0.5) ** 2 + (y - 0.45) ** 2 + (z - 0.5) ** 2) - 0.22
    P = np.zeros((5,) + phi.shape)
    P[0] = np.where(phi < 0, 1.2, 1000.0)
    P[2] = np.where(y < 0.25, 40.0, 0.0)
    P[4] = np.where(y < 0.25, 5e8, 1e5)
    full = m2c.Grid((n, n, n), h, (0,) * 6, (WATER, AIR), reinit_every=3, reinit_iters=2)
    full.set_prims(P, phi)
    full.step(20)
    full.sync()
    Ph, phih = P[..., n // 2:].copy(), phi[..., n // 2:].copy()
    g_or, ref, half, t = both(m2c, (n // 2, n, n), h, (S, 0, 0, 0, 0, 0), (WATER, AIR), Ph, phih, 20,
                              reinit=(3, 2))
    Wf = full.W.cpu().numpy()[..., n // 2:]
    Wh = half.W.cpu().numpy()
    assert max(rel_err(Wh, Wf)) <= 1e-12
    assert np.array_equal(half.phi.cpu().numpy() < 0, full.phi.cpu().numpy()[..., n // 2:] < 0)
    assert max(rel_err(Wh, ref.W)) <= TOL


@pytest.mark.parametrize("geom", [O.GEOM_SPHERICAL, O.GEOM_CYLINDRICAL])
def test_residual_with_geometry_and_mirrors_matches_oracle(m2c, geom):
    n = (64, 1, 1) if geom == O.GEOM_SPHERICAL else (48, 1, 36)
    bc = (S, 0, 0, 0, 0, 0) if geom == O.GEOM_SPHERICAL else (S, 0, 0, 0, S, 0)
    P, phi = WL.random_state(n, seed=13, eos=(WATER, AIR), two_phase=True)
    opts = dict(geom=geom, x0=0.0)
    g_or = O.Grid(n=n, h=1.0 / n[0], eos=(O.EOS(*WATER), O.EOS(*AIR)), bc=bc, **opts)
    R_ref, L_ref, st = O.residual(g_or, O.prims_to_cons(g_or, P, phi), phi)
    g = m2c.Grid(n, 1.0 / n[0], bc, (WATER, AIR), options=opts)
    g.set_prims(P, phi)
    R, L = g.residual()
    R, L = R.cpu().numpy(), L.cpu().numpy()
    assert max(rel_err(R, R_ref)) < 1e-11
    assert np.abs(L - L_ref).max() <= 1e-11 * max(np.abs(L_ref).max(), 1.0)


def test_mixed_precision_spherical_collapse_against_the_oracle(m2c):
    nr = 256
    h = 1.0 / nr
    r = (np.arange(nr) + 0.5) * h
    P, phi = bubble_in_water(r[None, None, :])
    opts = dict(geom=O.GEOM_SPHERICAL, x0=0.0)
    g_or, ref, g, t = both(m2c, (nr, 1, 1), h, (S, 0, 0, 0, 0, 0), (WATER, AIR), P, phi, 300, opts,
                           precision=1)
    Pg = O.cons_to_prims(g_or, g.W.cpu().numpy(), g.phi.cpu().numpy())
    Pr = O.cons_to_prims(g_or, ref.W, ref.phi)
    for v in (0, 4):
        assert np.abs(Pg[v] - Pr[v]).sum() / np.abs(Pr[v]).sum() <= 1e-4, v


def test_geometry_option_errors(m2c):
    g = m2c.Grid((16, 4, 1), 0.1, (S, 0, 0, 0, 0, 0), (AIR, AIR))
    for bad in (dict(geom=3), dict(geom=O.GEOM_SPHERICAL), dict(geom=O.GEOM_CYLINDRICAL),
                dict(geom=O.GEOM_CYLINDRICAL, x0=-1.0)):
        with pytest.raises(m2c.M2CError) as e:
            g.set_options(**bad)
        assert e.value.code == 1
    with pytest.raises(m2c.M2CError):
        g.set_tiling(16)  # a symmetry side runs the general kernel: 8-row tiles
