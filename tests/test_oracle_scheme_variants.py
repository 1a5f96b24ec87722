"""Pins of the oracle's scheme variants against what the mathematics fixes: the TVD RK3 and
forward Euler integrators and the constant time step of Sec. 4.3, the MC limiter of App. D
(Eq. theta) and the local Lax-Friedrichs flux of App. C.1 (Eq. Lax-Friedrichs). Orders of
accuracy in time and space, limiter invariants, flux consistency and symmetry, and convergence
to the exact two-stiffened-gas shock-tube solution. CPU only."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2508_16387_gb300 import workloads as WL

AIR = O.EOS(O.EOS_SG, (1.4, 0.0))
WATER = O.EOS(O.EOS_SG, (6.12, 3.43e8))


def _smooth_wave(nx, **scheme):
    """Density sine wave carried by u = 1 at p = 1 (perfect gas, periodic in x) and a positive
    smooth level set: both are translated exactly by the equations."""
    h = 1.0 / nx
    g = O.Grid(n=(nx, 1, 1), h=h, eos=(AIR, AIR), bc=(1, 1, 0, 0, 0, 0), reinit_every=10 ** 9, **scheme)
    x = (np.arange(nx) + 0.5) * h
    P = np.zeros((5, 1, 1, nx))
    P[0, 0, 0] = 1.0 + 0.2 * np.sin(2 * np.pi * x)
    P[1] = 1.0
    P[4] = 1.0
    phi = (0.5 + 0.3 * np.sin(2 * np.pi * x))[None, None, :]
    return g, x, P, phi


def _orders(errs):
    return [math.log2(a / b) for a, b in zip(errs, errs[1:])]


# --------------------------------------------------------------------------- time integration

@pytest.mark.parametrize("rk,lo,hi", [(1, 0.9, 1.3), (2, 1.9, 2.2), (3, 2.8, 3.5)])
def test_time_integrators_reach_their_order(rk, lo, hi):
    """On one fixed grid the spatial operator is the same for every time step, so the difference
    from a run with a 64x smaller constant time step is the time-integration error alone: it
    falls by 2^order per halving of dt (Sec. 4.3: forward Euler 1, TVD RK2 2, TVD RK3 3), for
    the conserved variables and for the level set. A wrong stage coefficient of RK3 leaves at
    most second order."""
    T, steps, ref_steps = 0.25, (40, 80, 160), 2560
    runs = {}
    for n in steps + (ref_steps,):
        g, _, P, phi = _smooth_wave(32, rk=rk, dt_fixed=T / n)
        W = O.prims_to_cons(g, P, phi)
        r = O.run(g, W, phi, n)
        assert r.t == pytest.approx(T, rel=1e-13) and np.all(r.dts == T / n)
        runs[n] = r
    ref = runs[ref_steps]
    eW = [np.abs(runs[n].W - ref.W).max() for n in steps]
    ephi = [np.abs(runs[n].phi - ref.phi).max() for n in steps]
    for errs in (eW, ephi):
        orders = _orders(errs)
        assert all(lo < o < hi for o in orders), orders


def test_forward_euler_converges_to_the_exact_translation():
    """Forward Euler (Sec. 4.3) with a CFL time step on the smooth translating wave: the density
    and the level set approach their exactly translated profiles at first order in h (the time
    error, dt ~ h, dominates), which a self-convergence test in dt alone cannot show (a wrong
    coefficient of the level-set update, planted in the oracle, converges there too)."""
    air = O.EOS(O.EOS_SG, (1.4, 0.0))
    u, T = 1.0, 0.25
    err_rho, err_phi = [], []
    for nx in (32, 64, 128):
        h = 1.0 / nx
        g = O.Grid(n=(nx, 1, 1), h=h, eos=(air, air), bc=(1, 1, 0, 0, 0, 0), reinit_every=10 ** 9, rk=1, cfl=0.2)
        x = (np.arange(nx) + 0.5) * h
        P = np.zeros((5, 1, 1, nx))
        P[0, 0, 0] = 1.0 + 0.2 * np.sin(2 * np.pi * x)
        P[1] = u
        P[4] = 1.0
        phi = (0.5 + 0.3 * np.sin(2 * np.pi * x))[None, None, :]
        W = O.prims_to_cons(g, P, phi)
        n = int(np.ceil(T / O.time_step(g, W, phi)))
        r = O.run(g, W, phi, n)
        Pn = O.cons_to_prims(g, r.W, r.phi)
        xs = x - u * r.t
        err_rho.append(np.abs(Pn[0, 0, 0] - (1.0 + 0.2 * np.sin(2 * np.pi * xs))).mean())
        err_phi.append(np.abs(r.phi[0, 0] - (0.5 + 0.3 * np.sin(2 * np.pi * xs))).mean())
    for errs in (err_rho, err_phi):
        orders = _orders(errs)
        assert min(orders) > 0.8, (orders, errs)


def test_constant_time_step_rejects_negative_values():
    g, _, P, phi = _smooth_wave(16, dt_fixed=-1.0)
    with pytest.raises(O.OracleError):
        O.run(g, O.prims_to_cons(O.Grid(n=g.n, h=g.h, eos=g.eos, bc=g.bc), P, phi), phi, 1)


# --------------------------------------------------------------------------- MC limiter

def test_mc_limiter_invariants():
    """App. D: phi(theta) = max(0, min(alpha theta, (theta + 1)/2, alpha)), sigma = phi b.
    alpha = 0 gives constant reconstruction; theta = 1 (linear data) keeps the central slope;
    the limiter is symmetric (sigma(a, b) = sigma(b, a)) and, for alpha in [1, 2], inside the
    second-order TVD region 0 <= sigma/b <= 2 min(theta, 1); zero at extrema."""
    rng = np.random.default_rng(11)
    for _ in range(2000):
        a, b = rng.normal(size=2) * 10.0 ** rng.uniform(-3, 3, size=2)
        alpha = rng.uniform(1.0, 2.0)
        s = O.mc_slope(a, b, alpha)
        assert O.mc_slope(a, b, 0.0) == 0.0
        assert s == pytest.approx(O.mc_slope(b, a, alpha), rel=1e-15, abs=0.0)
        if a * b <= 0.0:
            assert s == 0.0
        else:
            theta = a / b
            r = s / b
            assert -1e-15 <= r <= 2.0 * min(theta, 1.0) * (1 + 1e-15)
            assert s * b >= 0.0
    for b in (1e-3, 1.0, -7.5):
        assert O.mc_slope(b, b, 1.2) == b                 # linear data: central slope
        assert O.mc_slope(1e6 * b, b, 1.2) == 1.2 * b     # steep side: capped at alpha b
        assert O.mc_slope(1e-6 * b, b, 1.2) == pytest.approx(1.2e-6 * b, rel=1e-15)  # alpha a
    assert O.mc_slope(1.0, 0.0, 1.2) == 0.0 and O.mc_slope(0.0, 0.0, 1.2) == 0.0


# --------------------------------------------------------------------------- LLF flux

def _q(rho, u, v, w, p):
    return np.array([rho, u, v, w, p], float)


@pytest.mark.parametrize("eos,q", [(AIR, _q(1.2, 30.0, -4.0, 7.0, 1e5)), (WATER, _q(1000.0, -12.0, 3.0, 1.0, 2e8))])
def test_llf_consistency_mirror_and_rotation(eos, q):
    """Phi(W, W) is the physical flux (App. C.1; the HLLC flux, pinned consistent, gives the same);
    reflecting the normal velocity and swapping the sides negates the flux's mass and energy
    parts; the flux along y of a state with u and v swapped is the x flux with the momenta
    swapped."""
    for d in range(3):
        assert np.allclose(O.llf(eos, q, q, d), O.hllc(eos, q, q, d), rtol=1e-14, atol=0.0)
    qR = q * np.array([0.7, 1.3, 0.5, -1.0, 1.4])
    F = O.llf(eos, q, qR, 0)
    m = np.array([1.0, -1.0, 1.0, 1.0, 1.0])
    Fm = O.llf(eos, qR * m, q * m, 0)
    assert np.allclose(Fm, -F * m, rtol=1e-13, atol=1e-9 * np.abs(F).max())
    sw = [0, 2, 1, 3, 4]
    Fy = O.llf(eos, q[sw], qR[sw], 1)
    assert np.allclose(Fy[sw], F, rtol=1e-13, atol=1e-9 * np.abs(F).max())


MGW = O.EOS(O.EOS_MG, (1000.0, 1483.0, 1.75, 0.28, 0.0, -math.inf))


def _fd_c(eos, rho, p):
    """Sound speed from the thermodynamic identity c^2 = dp/drho|_e + p/rho^2 dp/de|_rho, both
    derivatives by central differences of p(rho, e) (independent of the oracle's c^2)."""
    e = O.energy(eos, rho, p)
    hr, he = 1e-7 * rho, 1e-7 * max(abs(e), 1.0)
    dpdr = (O.pressure(eos, rho + hr, e) - O.pressure(eos, rho - hr, e)) / (2 * hr)
    dpde = (O.pressure(eos, rho, e + he) - O.pressure(eos, rho, e - he)) / (2 * he)
    return math.sqrt(dpdr + p / rho ** 2 * dpde)


@pytest.mark.parametrize("eos,qL,qR", [
    (AIR, _q(1.2, 0.0, 0.0, 0.0, 1e5), _q(4.0, 0.0, 0.0, 0.0, 1e5)),          # contact at rest
    (AIR, _q(1.2, 150.0, 3.0, 0.0, 1e5), _q(2.5, -40.0, 0.0, 9.0, 3e5)),
    (MGW, _q(1010.0, 20.0, 0.0, 0.0, 3e7), _q(1040.0, -5.0, 1.0, 0.0, 6e7)),
])
def test_llf_dissipation_is_the_largest_eigenvalue(eos, qL, qR):
    """The mass component of Phi is (rho_L u_L + rho_R u_R)/2 - lambda (rho_R - rho_L)/2; the
    lambda it implies is the largest eigenvalue magnitude of the normal flux Jacobian,
    max(|u_L| + c_L, |u_R| + c_R) (App. C.1), with c from the thermodynamic identity."""
    F = O.llf(eos, qL, qR, 0)
    lam = (qL[0] * qL[1] + qR[0] * qR[1] - 2.0 * F[0]) / (qR[0] - qL[0])
    want = max(abs(qL[1]) + _fd_c(eos, qL[0], qL[4]), abs(qR[1]) + _fd_c(eos, qR[0], qR[4]))
    assert lam == pytest.approx(want, rel=1e-6)


# --------------------------------------------------------------------------- convergence

@pytest.mark.parametrize("scheme", [dict(limiter=O.LIM_MC), dict(flux=O.FLUX_LLF), dict(rk=3),
                                    dict(rk=3, limiter=O.LIM_MC, flux=O.FLUX_LLF)])
def test_variants_are_second_order_on_a_smooth_wave(scheme):
    """MUSCL with either limiter and either flux, with RK2 or RK3, is second order on the
    translated sine wave (App. D, App. C, Sec. 4.3); LLF, the more dissipative flux, has the
    larger error on the coarsest grid."""
    errs = []
    for nx in (32, 64, 128, 256):
        g, x, P, phi = _smooth_wave(nx, **scheme)
        W = O.prims_to_cons(g, P, phi)
        r = O.run(g, W, phi, int(math.ceil(0.5 / O.time_step(g, W, phi))))
        Pn = O.cons_to_prims(g, r.W, r.phi)
        errs.append(np.abs(Pn[0, 0, 0] - (1.0 + 0.2 * np.sin(2 * np.pi * (x - r.t)))).mean())
    orders = _orders(errs)
    assert min(orders) > 1.8 and math.log2(errs[0] / errs[-1]) / 3 > 1.9, orders
    if scheme.get("flux") == O.FLUX_LLF:
        g, x, P, phi = _smooth_wave(32)
        W = O.prims_to_cons(g, P, phi)
        r = O.run(g, W, phi, int(math.ceil(0.5 / O.time_step(g, W, phi))))
        Pn = O.cons_to_prims(g, r.W, r.phi)
        e_hllc = np.abs(Pn[0, 0, 0] - (1.0 + 0.2 * np.sin(2 * np.pi * (x - r.t)))).mean()
        assert errs[0] > 1.2 * e_hllc


@pytest.mark.parametrize("scheme", [dict(limiter=O.LIM_MC, rk=3), dict(flux=O.FLUX_LLF)])
def test_variants_converge_on_the_water_air_shock_tube(scheme):
    """Water | air shock tube (FIVER at the interface, the selected flux on both sides of it):
    the L1 error of density against the exact two-stiffened-gas solution decreases under
    refinement."""
    errs = []
    for nx in (64, 128, 256):
        s = WL.shock_tube(nx=nx, ny=1, nz=1)
        g = O.Grid(n=s.n, h=s.h, eos=tuple(O.EOS(*e) for e in s.eos), bc=s.bc, cfl=s.cfl,
                   reinit_every=s.reinit_every, reinit_iters=s.reinit_iters, **scheme)
        W = O.prims_to_cons(g, s.prims(), s.phi)
        r = O.run(g, W, s.phi, nx // 2)
        P = O.cons_to_prims(g, r.W, r.phi)
        x = (np.arange(nx) + 0.5) / nx
        ex, _ = O.exact_sample_sg(WATER.prm, (1000.0, 0.0, 1e9), AIR.prm, (1.0, 0.0, 1e5), (x - 0.5) / r.t)
        errs.append(np.abs(P[0, 0, 0] - ex[0]).mean() / np.abs(ex[0]).mean())
    assert errs[0] > errs[1] > errs[2], errs
    assert math.log2(errs[0] / errs[-1]) / 2 > 0.5, errs
