"""Pins of the oracle's Jones-Wilkins-Lee EOS (App. B.2, Eq. JWL_EOS with the sign of Reading
R35) and its wave curves (Reading R36) against what the mathematics fixes: the thermodynamic
identity for c^2, the inverse e(rho, p), the ideal-gas limit at low density, the
Rankine-Hugoniot jumps of its shocks, its rarefaction against an adaptive ODE integration, an
independent brute-force Riemann solution against air, and conservation in a stepped run.
CPU only."""
import math

import numpy as np
import pytest
from scipy.integrate import solve_ivp
from scipy.optimize import brentq

from oracle import oracle as O

# synthetic detonation-product parameters (omega, A1, A2, R1, R2, rho0)
JWL = O.EOS(O.EOS_JWL, (0.3, 4.0e11, 4.0e9, 4.5, 1.0, 1600.0))
AIR = O.EOS(O.EOS_SG, (1.4, 0.0))


def _fd_c2(eos, rho, p):
    e = O.energy(eos, rho, p)
    hr, he = 1e-7 * rho, 1e-7 * max(abs(e), 1.0)
    dpdr = (O.pressure(eos, rho + hr, e) - O.pressure(eos, rho - hr, e)) / (2 * hr)
    dpde = (O.pressure(eos, rho, e + he) - O.pressure(eos, rho, e - he)) / (2 * he)
    return dpdr + p / rho ** 2 * dpde


@pytest.mark.parametrize("rho,p", [(1600.0, 2e10), (1200.0, 5e9), (300.0, 1e8), (10.0, 1e6)])
def test_jwl_sound_speed_and_energy(rho, p):
    assert O.sound_speed2(JWL, rho, p) == pytest.approx(_fd_c2(JWL, rho, p), rel=1e-6)
    e = O.energy(JWL, rho, p)
    assert O.pressure(JWL, rho, e) == pytest.approx(p, rel=1e-12)


def test_jwl_is_an_ideal_gas_at_low_density():
    """Both exponential terms vanish as rho -> 0: p -> omega rho e and c^2 -> (1 + omega) p/rho,
    a perfect gas with gamma = 1 + omega."""
    w = JWL.prm[0]
    rho, e = 1e-3, 2e6
    assert O.pressure(JWL, rho, e) == pytest.approx(w * rho * e, rel=1e-12)
    p = w * rho * e
    assert O.sound_speed2(JWL, rho, p) == pytest.approx((1 + w) * p / rho, rel=1e-10)


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


@pytest.mark.parametrize("w,p", [((1600.0, 0.0, 2e10), 3e10), ((200.0, 50.0, 1e8), 2e9), ((5.0, 0.0, 1e6), 5e7)])
def test_jwl_shock_satisfies_the_jump_conditions(w, p):
    f, df, rs = O.wave_curve(JWL, w, p)
    assert rs > w[0]
    for res in _rh(JWL, w, (rs, w[1] - f, p)):
        assert res < 1e-11
    hp = 1e-5 * (p - w[2])   # f'(p) along the Hugoniot against a central difference of f
    fd = (O.wave_curve(JWL, w, p + hp)[0] - O.wave_curve(JWL, w, p - hp)[0]) / (2 * hp)
    assert df == pytest.approx(fd, rel=1e-7)


def _isentrope(eos, rho0, p0, p):
    """rho and f = integral of dp/(rho c) from p0 to p, adaptive DOP853 in p."""
    def rhs(q, y):
        c2 = O.sound_speed2(eos, y[0], q)
        return [1.0 / c2, 1.0 / (y[0] * math.sqrt(c2))]
    sol = solve_ivp(rhs, (p0, p), [rho0, 0.0], rtol=1e-13, atol=1e-16, method="DOP853")
    return sol.y[0, -1], sol.y[1, -1]


@pytest.mark.parametrize("w,p", [((1600.0, 0.0, 2e10), 1e9), ((1600.0, 0.0, 2e10), 1e5), ((300.0, 0.0, 1e8), 1e6)])
def test_jwl_rarefaction_matches_adaptive_integration(w, p):
    """Reading R36's RK4 in ln p (256 substeps per unit) against an adaptive DOP853 integration
    of the same isentrope ODE, over one to five decades of pressure."""
    f, df, rs = O.wave_curve(JWL, w, p)
    rho_ref, f_ref = _isentrope(JWL, w[0], w[2], p)
    assert rs == pytest.approx(rho_ref, rel=1e-10)
    assert f == pytest.approx(f_ref, rel=1e-10)
    assert df == pytest.approx(1.0 / (rs * math.sqrt(O.sound_speed2(JWL, rs, p))), rel=1e-12)


def _brute_force(wL, wR):
    """JWL (left) against air (right): shock branches from the Hugoniot energy equation by
    brentq, rarefaction branches by DOP853, the star pressure by brentq."""
    def side(eos, w, p, sgn, rho_hi):
        rho0, u0, p0 = w
        if p > p0:
            def H(r):
                return O.energy(eos, r, p) - O.energy(eos, rho0, p0) - 0.5 * (p + p0) * (1 / rho0 - 1 / r)
            r = brentq(H, rho0 * (1 + 1e-14), rho_hi * rho0, xtol=1e-300, rtol=1e-15)
            return u0 - sgn * math.sqrt((p - p0) * (1 / rho0 - 1 / r)), r
        r, f = _isentrope(eos, rho0, p0, p)
        return u0 - sgn * f, r

    air_hi = 6.0 * (1 - 1e-13)   # strong-shock compression limit (gamma + 1)/(gamma - 1) of air

    def F(p):
        return side(JWL, wL, p, 1, 30.0)[0] - side(AIR, wR, p, -1, air_hi)[0]
    hi = 2.0 * max(wL[2], wR[2])
    while F(hi) >= 0.0:   # F = u_L*(p) - u_R*(p) decreases with p
        hi *= 2.0
    ps = brentq(F, 1.0, hi, xtol=1e-300, rtol=1e-15)
    uL, rl = side(JWL, wL, ps, 1, 30.0)
    uR, rr = side(AIR, wR, ps, -1, air_hi)
    return ps, 0.5 * (uL + uR), rl, rr


@pytest.mark.parametrize("wL,wR", [
    ((1600.0, 0.0, 2e10), (1.2, 0.0, 1e5)),       # detonation products expanding into air
    ((50.0, 0.0, 5e7), (1.2, -200.0, 1e5)),       # weaker: products rarefaction, air shock
    ((10.0, 300.0, 1e6), (1.2, -300.0, 1e5)),     # collision: two shocks
])
def test_jwl_riemann_matches_brute_force(wL, wR):
    (ps, us, rl, rr), _ = O.riemann(JWL, wL, AIR, wR)
    bp, bu, brl, brr = _brute_force(wL, wR)
    assert ps == pytest.approx(bp, rel=1e-9)
    assert us == pytest.approx(bu, rel=1e-9)
    assert rl == pytest.approx(brl, rel=1e-9)
    assert rr == pytest.approx(brr, rel=1e-9)
    # mirror: the same problem with the sides swapped and the velocities negated
    (ps2, us2, rl2, rr2), _ = O.riemann(AIR, (wR[0], -wR[1], wR[2]), JWL, (wL[0], -wL[1], wL[2]))
    assert ps2 == pytest.approx(ps, rel=1e-12) and us2 == pytest.approx(-us, rel=1e-12)
    assert rl2 == pytest.approx(rr, rel=1e-12) and rr2 == pytest.approx(rl, rel=1e-12)


def test_jwl_periodic_run_conserves_and_keeps_uniform_flow():
    n = (10, 8, 6)
    shape = (n[2], n[1], n[0])
    g = O.Grid(n=n, h=0.01, eos=(JWL, AIR), bc=(1,) * 6)
    P = np.zeros((5,) + shape)
    P[0] = 1200.0
    P[1:4] = np.array([40.0, -20.0, 10.0])[:, None, None, None]
    P[4] = 5e9
    phi = np.ones(shape)
    W = O.prims_to_cons(g, P, phi)
    assert np.array_equal(O.run(g, W, phi, 4).W, W)
    rng = np.random.default_rng(9)
    P[0] = 1200.0 * (1 + 0.02 * rng.standard_normal(shape))
    P[4] = 5e9 * (1 + 0.05 * rng.standard_normal(shape))
    W = O.prims_to_cons(g, P, phi)
    r = O.run(g, W, phi, 10)
    for v in range(5):
        assert abs(r.W[v].sum() - W[v].sum()) <= 1e-13 * np.abs(W[v]).sum()
    assert not np.allclose(r.W[0], W[0])
