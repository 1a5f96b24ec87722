"""Pins of the oracle's narrow-band level set (Sec. 4.4: the level-set equation solved
in a band around the zero level set; Reading R38, the local level set of Peng et al.,
J. Comput. Phys. 155, 1999): the cutoff function's closed-form end conditions, a band
wider than the level set reproducing the full-domain method bit for bit, the values
beyond the outer tube clipped and held, and a sphere carried by a uniform flow whose
interface follows the full-domain one and the exact translation to within a small
fraction of a cell. CPU only."""
import numpy as np
import pytest

from oracle import oracle as O

AIR = O.EOS(O.EOS_SG, (1.4, 0.0))
WATER = O.EOS(O.EOS_SG, (6.12, 3.43e8))


def test_cutoff_closed_form():
    """c = 1 inside beta, 0 beyond gamma, C1 at both radii (zero slope), decreasing between,
    and c(|phi|) = (|phi| - gamma)^2 (2|phi| + gamma - 3 beta)/(gamma - beta)^3 at its midpoint."""
    beta, gamma, h = 3.0, 6.0, 0.01
    c = lambda x: O.band_cutoff(beta, gamma, h, x)  # noqa: E731
    assert c(0.0) == 1.0 and c(beta * h) == 1.0 and c(-beta * h) == 1.0
    assert c(gamma * h) == 0.0 and c(-7 * h) == 0.0
    eps = 1e-7 * h
    assert abs(c(beta * h + eps) - 1.0) < 1e-9
    assert abs(c(gamma * h - eps)) < 1e-9
    xs = np.linspace(beta * h, gamma * h, 101)
    vals = np.array([c(x) for x in xs])
    assert np.all(np.diff(vals) <= 0.0)
    assert c(4.5 * h) == pytest.approx(0.5, abs=1e-15)  # the cubic's symmetry point
    assert c(-4.5 * h) == c(4.5 * h)


def _bubble(n):
    h = 1.0 / n
    c = (np.arange(n) + 0.5) * h
    z, y, x = np.meshgrid(c, c, c, indexing="ij")
    phi = np.sqrt((x - 0.5) ** 2 + (y - 0.5) ** 2 + (z - 0.5) ** 2) - 0.2
    P = np.zeros((5,) + phi.shape)
    P[0] = np.where(phi < 0, 1.2, 1000.0)
    P[1] = np.where(x < 0.2, 200.0, 0.0)
    P[4] = np.where(x < 0.2, 5e8, 1e5)
    return h, P, phi


def test_a_band_wider_than_the_level_set_is_the_full_domain():
    """With beta above every |phi| of the run the cutoff is 1 and the clip does nothing: the same
    bits as the full-domain method, with FIVER, reinitialisation and phase updates at work."""
    n = 20
    h, P, phi = _bubble(n)
    full = O.Grid(n=(n, n, n), h=h, eos=(WATER, AIR), reinit_every=3, reinit_iters=2)
    band = O.Grid(n=(n, n, n), h=h, eos=(WATER, AIR), reinit_every=3, reinit_iters=2, band_beta=3 * n,
                  band_gamma=4 * n)
    W0 = O.prims_to_cons(full, P, phi)
    a = O.run(full, W0, phi, 12)
    b = O.run(band, W0, phi, 12)
    assert np.array_equal(a.W, b.W) and np.array_equal(a.phi, b.phi)


def test_values_beyond_the_outer_tube_are_clipped_and_held():
    """After a step every |phi| is at most gamma; cells that start beyond gamma hold exactly
    +-gamma (zero velocity there; the reinitialisation moves a plateau cell outwards and the clip
    puts it back), and the material map is unchanged by the clip."""
    n = 24
    h, P, phi = _bubble(n)
    gam = 5.0
    g = O.Grid(n=(n, n, n), h=h, eos=(WATER, AIR), reinit_every=1, reinit_iters=3, band_beta=2.0,
               band_gamma=gam)
    r = O.run(g, O.prims_to_cons(g, P, phi), phi, 6)
    assert np.abs(r.phi).max() <= gam * h
    far = np.abs(phi) > gam * h + 6 * 0.5 * h  # beyond any reach of 6 steps at CFL 0.5
    assert np.array_equal(r.phi[far], np.sign(phi[far]) * gam * h)
    g_full = O.Grid(n=(n, n, n), h=h, eos=(WATER, AIR), reinit_every=1, reinit_iters=3)
    rf = O.run(g_full, O.prims_to_cons(g_full, P, phi), phi, 6)
    assert np.array_equal(r.phi < 0, rf.phi < 0)


def _translated_sphere(band):
    """A sphere of radius 0.25 carried by a uniform flow of 300 m/s along (1, 1, 0)/sqrt(2) in a
    periodic box (one gas on both sides, so the flow stays exactly uniform), reinitialised every
    step, for 100 steps (about seven cells of travel)."""
    n = 32
    h = 1.0 / n
    c = (np.arange(n) + 0.5) * h
    z, y, x = np.meshgrid(c, c, c, indexing="ij")
    phi = np.sqrt((x - 0.4) ** 2 + (y - 0.4) ** 2 + (z - 0.5) ** 2) - 0.25
    P = np.zeros((5,) + phi.shape)
    P[0] = 1.0
    P[1] = P[2] = 300.0 / np.sqrt(2.0)
    P[4] = 1e5
    kw = dict(band_beta=3.0, band_gamma=6.0) if band else {}
    g = O.Grid(n=(n, n, n), h=h, eos=(AIR, AIR), bc=(1,) * 6, reinit_every=1, reinit_iters=5, **kw)
    r = O.run(g, O.prims_to_cons(g, P, phi), phi, 100)
    return h, x, y, z, r


def test_translating_sphere_follows_the_full_domain_and_the_exact_motion():
    h, x, y, z, rb = _translated_sphere(True)
    _, _, _, _, rf = _translated_sphere(False)
    near = np.abs(rf.phi) <= 1.5 * h
    assert np.abs(rb.phi[near] - rf.phi[near]).max() <= 0.02 * h
    assert np.array_equal(rb.phi < 0, rf.phi < 0)
    # the interior's centroid moves with the flow
    inside = rb.phi < 0
    s = 300.0 / np.sqrt(2.0) * rb.t
    assert s > 6 * h
    assert abs(x[inside].mean() - (0.4 + s)) <= 0.05 * h
    assert abs(y[inside].mean() - (0.4 + s)) <= 0.05 * h
    assert abs(z[inside].mean() - 0.5) <= 1e-12


def test_residual_is_the_full_domain_one_inside_beta_and_zero_beyond_gamma():
    """The level-set residual of one stage with the band: equal to the full-domain one (bit for
    bit) where |phi| <= beta, exactly zero where |phi| >= gamma, and in between of the same sign
    and a smaller magnitude that decreases with |phi|; the fluid residual is untouched."""
    n = 24
    h = 1.0 / n
    c = (np.arange(n) + 0.5) * h
    z, y, x = np.meshgrid(c, c, c, indexing="ij")
    phi = np.sqrt((x - 0.5) ** 2 + (y - 0.5) ** 2 + (z - 0.5) ** 2) - 0.2
    P = np.zeros((5,) + phi.shape)
    P[0] = np.where(phi < 0, 1.2, 1000.0)
    P[1] = 30.0
    P[2] = -20.0
    P[4] = 1e5
    kw = dict(n=(n, n, n), h=h, eos=(WATER, AIR), bc=(0,) * 6)
    gf, gb = O.Grid(**kw), O.Grid(band_beta=2.0, band_gamma=5.0, **kw)
    W = O.prims_to_cons(gf, P, phi)
    Rf, Lf, _ = O.residual(gf, W, phi)
    Rb, Lb, _ = O.residual(gb, W, phi)
    assert np.array_equal(Rf, Rb)
    a = np.abs(phi)
    inner, outer, taper = a <= 2 * h, a >= 5 * h, (a > 2 * h) & (a < 5 * h)
    assert np.array_equal(Lb[inner], Lf[inner])
    assert np.all(Lb[outer] == 0.0)
    moving = taper & (np.abs(Lf) > 0)
    assert moving.sum() > 100
    ratio = Lb[moving] / Lf[moving]
    assert np.all((ratio > 0.0) & (ratio < 1.0))
    order = np.argsort(a[moving])
    assert np.all(np.diff(ratio[order]) <= 1e-15)
