"""Pins of the oracle's spherical and cylindrical symmetry forms (Sec. 3.4, Eqs.
euler1d_spherical and Euler_cylindrical, Reading R37) and of its symmetry (mirror) boundary:
a half domain with a mirror side equals the mirror-symmetric full domain; the 1D spherical and
2D cylindrical forms converge to the 3D Cartesian solution of a spherical shock tube (computed
by the plain 3D scheme on an octant with mirror sides), while the planar 1D form does not. CPU
only."""
import numpy as np
import pytest

from oracle import oracle as O

AIR = O.EOS(O.EOS_SG, (1.4, 0.0))
WATER = O.EOS(O.EOS_SG, (6.12, 3.43e8))


def _advance(g, W, phi, T):
    """Whole CFL steps until t >= T (the last one overshoots by less than one step)."""
    t, n = 0.0, 0
    while t < T:
        r = O.run(g, W, phi, 1, step0=n, t0=t)
        W, phi, t, n = r.W, r.phi, r.t, n + 1
    return W, phi, t


def _sod(r):
    """Spherical shock tube: (rho, p) = (1, 10) for r < 0.2, (0.125, 1) outside, at rest."""
    P = np.zeros((5,) + r.shape)
    P[0] = np.where(r < 0.2, 1.0, 0.125)
    P[4] = np.where(r < 0.2, 10.0, 1.0)
    return P


T_END = 0.06


def _radial_1d(nr, geom):
    h = 0.5 / nr
    g = O.Grid(n=(nr, 1, 1), h=h, eos=(AIR, AIR), bc=(O.BC_SYMMETRY, 0, 0, 0, 0, 0), geom=geom,
               reinit_every=10 ** 9)
    r = (np.arange(nr) + 0.5) * h
    phi = np.ones((1, 1, nr))
    W, phi, _ = _advance(g, O.prims_to_cons(g, _sod(r)[:, None, None, :], phi), phi, T_END)
    return r, O.cons_to_prims(g, W, phi)[0, 0, 0]


@pytest.fixture(scope="module")
def spherical_reference():
    return _radial_1d(400, O.GEOM_SPHERICAL)


def _octant_3d(m):
    h = 0.5 / m
    S = O.BC_SYMMETRY
    g = O.Grid(n=(m, m, m), h=h, eos=(AIR, AIR), bc=(S, 0, S, 0, S, 0), reinit_every=10 ** 9)
    c = (np.arange(m) + 0.5) * h
    z, y, x = np.meshgrid(c, c, c, indexing="ij")
    r = np.sqrt(x * x + y * y + z * z)
    phi = np.ones(r.shape)
    W, phi, _ = _advance(g, O.prims_to_cons(g, _sod(r), phi), phi, T_END)
    return r, O.cons_to_prims(g, W, phi)[0]


def test_spherical_form_converges_to_the_3d_solution(spherical_reference):
    """The 3D Cartesian octant (no source term; the sphere's symmetry from three mirror sides)
    approaches the fine 1D spherical solution as it is refined, and stays far from the planar 1D
    solution (the same 1D grid without the source term)."""
    r1, rho1 = spherical_reference
    rp, rhop = _radial_1d(400, O.GEOM_CARTESIAN)
    errs, errs_planar = [], []
    for m in (16, 24, 32):
        r3, rho3 = _octant_3d(m)
        mask = r3 < 0.45
        errs.append(np.abs(rho3 - np.interp(r3, r1, rho1))[mask].mean())
        errs_planar.append(np.abs(rho3 - np.interp(r3, rp, rhop))[mask].mean())
    assert errs[0] > errs[1] > errs[2], errs
    assert errs[2] < 0.01, errs
    assert min(errs_planar) > 4 * errs[2], (errs, errs_planar)


def test_cylindrical_form_converges_to_the_spherical_one(spherical_reference):
    """The same sphere on the (r, z) half plane of the cylindrical form (mirror sides at r = 0
    and z = 0) approaches the 1D spherical solution along r_s = sqrt(r^2 + z^2)."""
    r1, rho1 = spherical_reference
    errs = []
    for m in (16, 32, 64):
        h = 0.5 / m
        S = O.BC_SYMMETRY
        g = O.Grid(n=(m, 1, m), h=h, eos=(AIR, AIR), bc=(S, 0, 0, 0, S, 0), geom=O.GEOM_CYLINDRICAL,
                   reinit_every=10 ** 9)
        c = (np.arange(m) + 0.5) * h
        z, x = np.meshgrid(c, c, indexing="ij")
        rs = np.sqrt(x * x + z * z)[:, None, :]
        phi = np.ones(rs.shape)
        W, phi, _ = _advance(g, O.prims_to_cons(g, _sod(rs), phi), phi, T_END)
        rho = O.cons_to_prims(g, W, phi)[0]
        mask = rs < 0.45
        errs.append(np.abs(rho - np.interp(rs, r1, rho1))[mask].mean())
    assert errs[0] > errs[1] > errs[2], errs
    assert errs[2] < 0.006, errs


def test_spherical_rest_state_stays_at_rest():
    """At rest the source vanishes and a uniform pressure exerts no net force."""
    g = O.Grid(n=(32, 1, 1), h=0.01, eos=(AIR, AIR), bc=(O.BC_SYMMETRY, 0, 0, 0, 0, 0),
               geom=O.GEOM_SPHERICAL, x0=0.0)
    P = np.zeros((5, 1, 1, 32))
    P[0] = 1.3
    P[4] = 2e5
    phi = np.ones((1, 1, 32))
    W = O.prims_to_cons(g, P, phi)
    assert np.array_equal(O.run(g, W, phi, 5).W, W)


def _mirror_problem(n):
    """A water/air problem symmetric about the planes x = 1/2 and z = 1/2 (an air bubble centred
    on both, a pressure step along y)."""
    h = 1.0 / n
    c = (np.arange(n) + 0.5) * h
    z, y, x = np.meshgrid(c, c, c, indexing="ij")
    phi = np.sqrt((x - 0.5) ** 2 + (y - 0.45) ** 2 + (z - 0.5) ** 2) - 0.22
    P = np.zeros((5,) + phi.shape)
    P[0] = np.where(phi < 0, 1.2, 1000.0)
    P[2] = np.where(y < 0.25, 40.0, 0.0)
    P[4] = np.where(y < 0.25, 5e8, 1e5)
    return h, P, phi


@pytest.fixture(scope="module")
def mirror_full_run():
    n = 16
    h, P, phi = _mirror_problem(n)
    full = O.Grid(n=(n, n, n), h=h, eos=(WATER, AIR), bc=(0,) * 6, reinit_every=3, reinit_iters=2)
    return n, h, P, phi, O.run(full, O.prims_to_cons(full, P, phi), phi, 8)


@pytest.mark.parametrize("axis,side", [("x", "lo"), ("x", "hi"), ("z", "lo"), ("z", "hi")])
def test_mirror_side_equals_the_symmetric_full_domain(mirror_full_run, axis, side):
    """The half domain on one side of a symmetry plane, with a mirror side on that plane (its
    lower side for the upper half, its upper side for the lower half, along x or z), reproduces
    the full domain's half, FIVER faces on the mirror plane included."""
    n, h, P, phi, rf = mirror_full_run
    m = n // 2
    half_sel = slice(m, None) if side == "lo" else slice(None, m)
    if axis == "x":
        sel = (Ellipsis, half_sel)
        shape = (m, n, n)
        bc = [0] * 6
        bc[0 if side == "lo" else 1] = O.BC_SYMMETRY
    else:
        sel = (Ellipsis, half_sel, slice(None), slice(None))
        shape = (n, n, m)
        bc = [0] * 6
        bc[4 if side == "lo" else 5] = O.BC_SYMMETRY
    half = O.Grid(n=shape, h=h, eos=(WATER, AIR), bc=tuple(bc), reinit_every=3, reinit_iters=2)
    Ph, phih = P[sel].copy(), phi[sel].copy()
    rh = O.run(half, O.prims_to_cons(half, Ph, phih), phih, 8)
    assert rf.stats["interface_faces"] > 0
    assert rh.t == pytest.approx(rf.t, rel=1e-13)
    for v in range(5):
        a, b = rh.W[v], rf.W[v][sel]
        assert np.abs(a - b).max() <= 1e-12 * np.abs(rf.W[v]).max(), v
    assert np.array_equal(rh.phi < 0, rf.phi[sel] < 0)


def _steady_radial_flow(r, alpha, gamma=1.4):
    """Isentropic steady radial flow of a perfect gas through (rho, u, p) = (1, 50, 1e5) at
    r = 1 (subsonic branch): rho u r^alpha = m, p = K rho^gamma and the Bernoulli sum
    gamma/(gamma - 1) p/rho + u^2/2 = H, each density by scipy's brentq. It is a steady solution
    of the spherical (alpha = 2) or cylindrical (alpha = 1) Euler equations of Sec. 3.4."""
    from scipy.optimize import brentq
    m, K = 50.0, 1e5
    H = gamma / (gamma - 1.0) * 1e5 + 0.5 * 50.0 ** 2
    out = []
    for ri in r:
        def bern(rho):
            return gamma / (gamma - 1.0) * K * rho ** (gamma - 1.0) + 0.5 * (m / (rho * ri ** alpha)) ** 2 - H
        rho_sonic = (m ** 2 / (gamma * K * ri ** (2 * alpha))) ** (1.0 / (gamma + 1.0))
        rho = brentq(bern, rho_sonic * (1.0 + 1e-9), 10.0, xtol=1e-15, rtol=1e-15)
        out.append((rho, m / (rho * ri ** alpha), K * rho ** gamma))
    return np.array(out).T


@pytest.mark.parametrize("geom,alpha", [(O.GEOM_SPHERICAL, 2), (O.GEOM_CYLINDRICAL, 1)])
def test_steady_radial_flow_residual_vanishes_at_second_order(geom, alpha):
    """The stage residual of the exact steady radial flow on r in [1, 1.5] falls at second order
    under refinement (away from the ends): the flux differences and the geometric source
    -(alpha/r) u_r (rho, rho u, rho v, rho w, rho E + p) of Sec. 3.4, taken at the cell centre
    r = x0 + (i + 1/2) h (Reading R37), balance to O(h^2). A source taken half a cell off the
    centre, planted in the oracle, leaves an O(h) residual and fails it."""
    errs = []
    for nr in (32, 64, 128):
        h = 0.5 / nr
        g = O.Grid(n=(nr, 1, 1), h=h, eos=(AIR, AIR), geom=geom, x0=1.0, reinit_every=10 ** 9)
        r = 1.0 + (np.arange(nr) + 0.5) * h
        rho, u, p = _steady_radial_flow(r, alpha)
        P = np.zeros((5, 1, 1, nr))
        P[0, 0, 0], P[1, 0, 0], P[4, 0, 0] = rho, u, p
        phi = np.ones((1, 1, nr))
        R, _, _ = O.residual(g, O.prims_to_cons(g, P, phi), phi)
        inner = slice(3, nr - 3)
        errs.append([np.abs(R[v, 0, 0, inner]).max() for v in (0, 1, 4)])
    errs = np.array(errs)
    orders = np.log2(errs[:-1] / errs[1:])   # rows: refinements; columns: mass, momentum, energy
    assert orders.min() > 1.7 and orders[-1].min() > 1.85, orders


@pytest.mark.parametrize("mirror", [True, False])
def test_phase_update_across_a_mirror_side(mirror):
    """A cell on the x- side that becomes water with no water face neighbour takes the mean of
    its 26-neighbourhood's water cells (Reading R17). Its only water neighbour, an edge neighbour
    in the plane of the side, appears twice: itself, and its image across the side. With a
    mirror side the image's normal velocity is negated, so the mean has u = 0, as the symmetry
    demands; with a transmissive side the image is an unchanged copy and u stays."""
    n = (4, 4, 4)
    bc = (O.BC_SYMMETRY if mirror else 0, 0, 0, 0, 0, 0)
    g = O.Grid(n=n, h=0.25, eos=(WATER, AIR), bc=bc)
    P = np.zeros((5, 4, 4, 4))
    P[0], P[4] = 1.2, 1e5                     # air everywhere ...
    phi = -np.ones((4, 4, 4))
    P[:, 2, 2, 0] = (1000.0, 30.0, 5.0, -7.0, 2e5)  # ... but one water cell at (i, j, k) = (0, 2, 2)
    phi[2, 2, 0] = 1.0
    W = O.prims_to_cons(g, P, phi)
    id_old = (phi < 0).astype(np.uint8)
    phi_new = phi.copy()
    phi_new[1, 1, 0] = 0.5                    # cell (0, 1, 1) becomes water
    W2, phi2, nflip = O.phase_fix(g, W, phi_new, id_old)
    assert nflip == 1
    q = O.cons_to_prims(g, W2, phi2)[:, 1, 1, 0]
    assert q[0] == pytest.approx(1000.0, rel=1e-14) and q[4] == pytest.approx(2e5, rel=1e-12)
    assert q[2] == pytest.approx(5.0, rel=1e-12) and q[3] == pytest.approx(-7.0, rel=1e-12)
    assert abs(q[1] - (0.0 if mirror else 30.0)) <= 1e-12 * 30.0
