"""Pins of the oracle's Noble-Abel stiffened gas (Sec. 3.3, Eq. NASG_EOS) against what the
mathematics fixes: the thermodynamic identity for c^2, the inverse e(rho, p), the reduction to
the stiffened gas at b = 0, the Rankine-Hugoniot jumps of its shocks, the isentrope and the
Riemann invariant across its rarefactions, an independent brute-force Riemann solution, and
conservation in a stepped two-material run. CPU only."""
import math

import numpy as np
import pytest
from scipy.integrate import solve_ivp
from scipy.optimize import brentq

from oracle import oracle as O

# synthetic liquid-like and gas-like parameter sets (gamma, p_c, b, e_c)
LIQ = O.EOS(O.EOS_NASG, (1.5, 5.0e8, 5.0e-4, -1.0e6))
GAS = O.EOS(O.EOS_NASG, (1.4, 0.0, 1.0e-3, 0.0))
AIR = O.EOS(O.EOS_SG, (1.4, 0.0))


def _fd_c2(eos, rho, p):
    """c^2 = dp/drho|_e + p/rho^2 dp/de|_rho (App. C.2) by central differences of p(rho, e)."""
    e = O.energy(eos, rho, p)
    hr, he = 1e-7 * rho, 1e-7 * max(abs(e), 1.0)
    dpdr = (O.pressure(eos, rho + hr, e) - O.pressure(eos, rho - hr, e)) / (2 * hr)
    dpde = (O.pressure(eos, rho, e + he) - O.pressure(eos, rho, e - he)) / (2 * he)
    return dpdr + p / rho ** 2 * dpde


@pytest.mark.parametrize("eos,rho,p", [(LIQ, 1000.0, 1e5), (LIQ, 1200.0, 2e9), (LIQ, 900.0, -2e8),
                                       (GAS, 1.2, 1e5), (GAS, 300.0, 5e8)])
def test_nasg_sound_speed_and_energy(eos, rho, p):
    assert O.sound_speed2(eos, rho, p) == pytest.approx(_fd_c2(eos, rho, p), rel=1e-6)
    e = O.energy(eos, rho, p)
    assert O.pressure(eos, rho, e) == pytest.approx(p, rel=1e-12, abs=1e-6 * abs(eos.prm[1]) + 1e-9)


def test_nasg_covolume_bounds_the_density():
    """rho b < 1 is the EOS domain: the pressure at fixed e grows without bound towards it."""
    e = 1e6
    ps = [O.pressure(LIQ, (1.0 - x) / LIQ.prm[2], e) for x in (1e-1, 1e-2, 1e-3)]
    assert ps[0] < ps[1] < ps[2] and ps[2] > 100 * ps[0]
    with pytest.raises(O.OracleError):
        O.pressure(LIQ, 1.0 / LIQ.prm[2], e)


@pytest.mark.parametrize("wL,wR", [((1000.0, 0.0, 1e9), (1.0, 0.0, 1e5)), ((1000.0, 300.0, 1e5), (1.2, -100.0, 1e5)),
                                   ((1000.0, -50.0, 1e6), (1.2, 200.0, 1e5))])
def test_nasg_without_covolume_is_the_stiffened_gas(wL, wR):
    """b = 0: the same Riemann solution as the stiffened gas with the same gamma and p_c, whatever
    e_c (a constant shift of the internal energy does not enter the wave curves)."""
    sg = O.EOS(O.EOS_SG, (1.5, 5.0e8))
    for ec in (0.0, -1.0e6, 3.0e5):
        nasg = O.EOS(O.EOS_NASG, (1.5, 5.0e8, 0.0, ec))
        a, _ = O.riemann(nasg, wL, AIR, wR)
        b, _ = O.riemann(sg, wL, AIR, wR)
        assert np.allclose(a, b, rtol=1e-13, atol=1e-12)


@pytest.mark.parametrize("u", [50.0, 100.0, 300.0])
def test_nasg_without_covolume_is_the_stiffened_gas_in_tension(u):
    """Two liquid states separating at +-u: with b = 0 the star pressure falls below zero (into
    tension, above the lowest admissible pressure -p_c of both EOS) and is the stiffened gas's,
    whatever e_c; a lower bound of 0 for NASG, planted in the oracle, fails it."""
    sg = O.EOS(O.EOS_SG, (1.5, 5.0e8))
    wl, wr = (1000.0, -u, 1e5), (1000.0, u, 1e5)
    b, _ = O.riemann(sg, wl, sg, wr)
    assert -5.0e8 < b[0] < 0.0
    for ec in (0.0, -1.0e6):
        nasg = O.EOS(O.EOS_NASG, (1.5, 5.0e8, 0.0, ec))
        a, _ = O.riemann(nasg, wl, nasg, wr)
        assert np.allclose(a, b, rtol=1e-13, atol=1e-12)


def _rh(eos, ahead, behind):
    r0, u0, p0 = ahead
    r1, u1, p1 = behind
    S = (r1 * u1 - r0 * u0) / (r1 - r0)
    m0, m1 = r0 * (u0 - S), r1 * (u1 - S)
    e0, e1 = O.energy(eos, r0, p0), O.energy(eos, r1, p1)
    mom = (m0 * (u0 - S) + p0) - (m1 * (u1 - S) + p1)
    en = (m0 * (e0 + 0.5 * (u0 - S) ** 2) + p0 * (u0 - S)) - (m1 * (e1 + 0.5 * (u1 - S) ** 2) + p1 * (u1 - S))
    return (abs(m0 - m1) / abs(m0), abs(mom) / (abs(m0 * (u0 - S)) + abs(p0) + abs(p1)),
            abs(en) / (abs(m0 * (e0 + 0.5 * (u0 - S) ** 2)) + abs(p0 * (u0 - S)) + abs(p1 * (u1 - S))))


@pytest.mark.parametrize("eos,w,p", [(LIQ, (1000.0, 10.0, 1e5), 3e9), (GAS, (1.2, 0.0, 1e5), 2e6)])
def test_nasg_shock_satisfies_the_jump_conditions(eos, w, p):
    f, df, rs = O.wave_curve(eos, w, p)
    # the left-facing wave through w: the state behind it is (rs, u - f, p)
    for res in _rh(eos, w, (rs, w[1] - f, p)):
        assert res < 1e-11
    hp = 1e-5 * (p - w[2])   # f'(p) along the Hugoniot against a central difference of f
    fd = (O.wave_curve(eos, w, p + hp)[0] - O.wave_curve(eos, w, p - hp)[0]) / (2 * hp)
    assert df == pytest.approx(fd, rel=1e-7)


@pytest.mark.parametrize("eos,w,p", [(LIQ, (1000.0, 10.0, 3e8), 1e5), (GAS, (1.2, 0.0, 1e5), 2e3)])
def test_nasg_rarefaction_keeps_isentrope_and_riemann_invariant(eos, w, p):
    """Across a rarefaction (p + p_c)(1/rho - b)^gamma and u + 2 c (1 - rho b)/(gamma - 1) are
    constant (the left wave: u behind = u - f)."""
    g, pc, b, _ = eos.prm
    f, df, rs = O.wave_curve(eos, w, p)
    assert (p + pc) * (1 / rs - b) ** g == pytest.approx((w[2] + pc) * (1 / w[0] - b) ** g, rel=1e-12)

    def J(rho, u, pp):
        return u + 2 * math.sqrt(O.sound_speed2(eos, rho, pp)) * (1 - rho * b) / (g - 1)
    assert J(rs, w[1] - f, p) == pytest.approx(J(*w), rel=1e-12)
    # f' = 1/(rho c) behind the wave
    assert df == pytest.approx(1.0 / (rs * math.sqrt(O.sound_speed2(eos, rs, p))), rel=1e-12)


def _brute_force(eosL, wL, eosR, wR):
    """Shock branches: the Hugoniot energy equation solved by brentq with the oracle's e(rho, p);
    rarefaction branches: d rho/dp = 1/c^2 and du = -dp/(rho c) integrated by scipy DOP853;
    the star pressure by brentq."""
    def side(eos, w, p, sgn):
        rho0, u0, p0 = w
        if p > p0:
            def H(r):
                return O.energy(eos, r, p) - O.energy(eos, rho0, p0) - 0.5 * (p + p0) * (1 / rho0 - 1 / r)
            b = eos.prm[2]
            r = brentq(H, rho0 * (1 + 1e-14), (1 - 1e-12) / b if b > 0 else 1e9 * rho0, xtol=1e-300, rtol=1e-15)
            return u0 - sgn * math.sqrt((p - p0) * (1 / rho0 - 1 / r)), r

        def rhs(q, y):
            c2 = O.sound_speed2(eos, y[0], q)
            return [1.0 / c2, 1.0 / (y[0] * math.sqrt(c2))]
        sol = solve_ivp(rhs, (p0, p), [rho0, 0.0], rtol=1e-13, atol=1e-14, method="DOP853")
        return u0 - sgn * sol.y[1, -1], sol.y[0, -1]

    def F(p):
        return side(eosL, wL, p, 1)[0] - side(eosR, wR, p, -1)[0]
    lo = max(-eosL.prm[1], -eosR.prm[1]) + 1.0
    ps = brentq(F, lo, 1e11, xtol=1e-300, rtol=1e-15)
    uL, rl = side(eosL, wL, ps, 1)
    uR, rr = side(eosR, wR, ps, -1)
    return ps, 0.5 * (uL + uR), rl, rr


@pytest.mark.parametrize("wL,wR,eosL,eosR", [
    ((1000.0, 0.0, 1e9), (1.2, 0.0, 1e5), LIQ, GAS),        # liquid rarefaction, gas shock
    ((1000.0, 300.0, 1e5), (1.2, -100.0, 1e5), LIQ, GAS),   # collision: two shocks
    ((1000.0, -50.0, 1e6), (1.2, 200.0, 1e5), LIQ, GAS),    # expansion: two rarefactions
    ((1.2, 0.0, 1e5), (1000.0, 0.0, 1e9), GAS, LIQ),        # mirrored roles
])
def test_nasg_riemann_matches_brute_force(wL, wR, eosL, eosR):
    (ps, us, rl, rr), _ = O.riemann(eosL, wL, eosR, wR)
    bp, bu, brl, brr = _brute_force(eosL, wL, eosR, wR)
    assert ps == pytest.approx(bp, rel=1e-9)
    assert us == pytest.approx(bu, rel=1e-9, abs=1e-9 * (abs(wL[1]) + abs(wR[1]) + 1.0))
    assert rl == pytest.approx(brl, rel=1e-9)
    assert rr == pytest.approx(brr, rel=1e-9)


def test_nasg_two_material_periodic_run_conserves_and_keeps_uniform_flow():
    """A periodic 3D run with a NASG liquid and an SG gas: mass, momentum and energy are conserved
    to rounding in a single-material box and a uniform flow stays uniform bit for bit."""
    n = (10, 8, 6)
    shape = (n[2], n[1], n[0])
    g = O.Grid(n=n, h=0.1, eos=(LIQ, AIR), bc=(1,) * 6)
    P = np.zeros((5,) + shape)
    P[0] = 1000.0
    P[1:4] = np.array([3.0, -2.0, 1.0])[:, None, None, None]
    P[4] = 2e7
    phi = np.ones(shape)
    W = O.prims_to_cons(g, P, phi)
    r = O.run(g, W, phi, 4)
    assert np.array_equal(r.W, W)
    rng = np.random.default_rng(5)
    P[0] = 1000.0 * (1 + 0.02 * rng.standard_normal(shape))
    P[4] = 2e7 * (1 + 0.05 * rng.standard_normal(shape))
    W = O.prims_to_cons(g, P, phi)
    r = O.run(g, W, phi, 10)
    for v in range(5):
        assert abs(r.W[v].sum() - W[v].sum()) <= 1e-13 * np.abs(W[v]).sum()
    assert not np.allclose(r.W[0], W[0])
