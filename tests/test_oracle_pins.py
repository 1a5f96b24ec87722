"""Pins of the CPU FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: a value the
paper prints, a closed form, a conservation law, an invariant, a symmetry, a
library routine (scipy) or convergence to the exact solution. None of them
touches the GPU.
"""
import json
import math
import os

import numpy as np
import pytest
from scipy.integrate import solve_ivp

from oracle import oracle as O
from paper_2508_16387_gb300 import workloads as WL

HERE = os.path.dirname(os.path.abspath(__file__))

WATER = O.EOS(O.EOS_SG, (6.12, 3.43e8))
AIR = O.EOS(O.EOS_SG, (1.4, 0.0))
MGW = O.EOS(O.EOS_MG, (1000.0, 1483.0, 1.75, 0.28, 0.0, -math.inf))
MGW_CUT = O.EOS(O.EOS_MG, (1000.0, 1483.0, 1.75, 0.28, 0.0, -0.05))


def _fd_c2(eos, rho, p):
    """c^2 from the thermodynamic identity c^2 = dp/drho|_e + p/rho^2 dp/de|_rho (App. C.2),
    with both partial derivatives taken by central differences of the oracle's p(rho, e)."""
    e = O.energy(eos, rho, p)
    hr = 1e-8 * rho
    he = 1e-8 * max(abs(e), 1.0)
    dpdr = (O.pressure(eos, rho + hr, e) - O.pressure(eos, rho - hr, e)) / (2 * hr)
    dpde = (O.pressure(eos, rho, e + he) - O.pressure(eos, rho, e - he)) / (2 * he)
    return dpdr + p / rho ** 2 * dpde


# --------------------------------------------------------------------------- EOS

@pytest.mark.parametrize("eos,rho,p", [
    (WATER, 1000.0, 1e5), (WATER, 1200.0, 1e9), (AIR, 1.2, 1e5), (AIR, 5.0, 3e6),
    (MGW, 1000.0, 1e5), (MGW, 1243.0, 1e9), (MGW, 990.0, -1e6), (MGW_CUT, 940.0, -1e7),
])
def test_sound_speed_matches_thermodynamic_identity(eos, rho, p):
    assert O.sound_speed2(eos, rho, p) == pytest.approx(_fd_c2(eos, rho, p), rel=1e-5)


@pytest.mark.parametrize("eos,rho,p", [(WATER, 1100.0, 3e8), (MGW, 1100.0, 3e8), (MGW, 980.0, -2e6), (AIR, 2.0, 4e5)])
def test_energy_inverts_pressure(eos, rho, p):
    e = O.energy(eos, rho, p)
    assert O.pressure(eos, rho, e) == pytest.approx(p, rel=1e-13, abs=1e-6)


def test_perfect_gas_and_stiffened_gas_closed_forms():
    # NASG with b = e_c = 0 (Sec. 3.3): p = (gamma - 1) rho e - gamma p_c
    assert O.pressure(AIR, 1.3, 2.0e5) == pytest.approx(0.4 * 1.3 * 2.0e5, rel=1e-15)
    assert O.pressure(WATER, 1000.0, 4.2e5) == pytest.approx(5.12 * 1000.0 * 4.2e5 - 6.12 * 3.43e8, rel=1e-14)


def test_mg_reference_state_sound_speed_is_c0():
    # At eta = 0, e = e0 the MG pressure is 0 and the sound speed is c0 (App. B.3).
    assert O.pressure(MGW, 1000.0, 0.0) == 0.0
    assert math.sqrt(O.sound_speed2(MGW, 1000.0, 0.0)) == pytest.approx(1483.0, rel=1e-14)


@pytest.mark.parametrize("eos,rho_c", [(MGW, 1000.0), (MGW_CUT, 1000.0 / 1.05)])
def test_mg_branches_join_continuously(eos, rho_c):
    # K0 = rho0 c0^2 makes p_R and its derivative continuous at eta = 0; at eta_min the
    # cutoff branch starts from p_min = K0 eta_min with continuous e_R (App. B.3). A jump
    # would keep p(rho_c + eps) - p(rho_c - eps) finite as eps -> 0; continuity makes it O(eps).
    e = 500.0
    jumps = []
    for eps in (1e-4 * rho_c, 1e-5 * rho_c):
        jumps.append(abs(O.pressure(eos, rho_c + eps, e) - O.pressure(eos, rho_c - eps, e)))
    assert jumps[1] < 0.11 * jumps[0]
    if eos is MGW:
        # C^1 at eta = 0: the one-sided slopes agree
        h = 1e-4
        p0 = O.pressure(eos, rho_c, e)
        sl = (p0 - O.pressure(eos, rho_c - h, e)) / h
        sr = (O.pressure(eos, rho_c + h, e) - p0) / h
        assert sl == pytest.approx(sr, rel=1e-3)


# --------------------------------------------------------------------------- limiter

def test_van_albada_special_values():
    rng = np.random.default_rng(0)
    for a, b in rng.uniform(-3, 3, size=(200, 2)):
        s = O.va_slope(a, b)
        assert s == O.va_slope(b, a)                      # symmetric limiter
        if a * b <= 0:
            assert s == 0.0                               # modified VA: no slope at extrema
        else:
            theta = a / b
            phi = (theta ** 2 + theta) / (theta ** 2 + 1.0)  # App. D, Eq. vanalbada, A = B = 1, k = 2
            assert s == pytest.approx(phi * b, rel=1e-13)
            assert 0.0 <= s / b <= 2.0 and 0.0 <= s / a <= 2.0  # inside the TVD region
    assert O.va_slope(0.7, 0.7) == 0.7                    # linear data keeps its slope
    assert O.va_slope(0.0, 1.0) == 0.0


# --------------------------------------------------------------------------- HLLC

def _phys_flux(eos, q, d):
    rho, u, v, w, p = q
    e = O.energy(eos, rho, p)
    E = e + 0.5 * (u * u + v * v + w * w)
    vel = [u, v, w]
    un = vel[d]
    F = np.array([rho * un, rho * un * u, rho * un * v, rho * un * w, (rho * E + p) * un])
    F[1 + d] += p
    return F


@pytest.mark.parametrize("eos", [WATER, AIR, MGW])
def test_hllc_consistency(eos):
    rng = np.random.default_rng(1)
    base = (1000.0, 1e8) if eos is not AIR else (1.2, 1e5)
    for _ in range(20):
        q = [base[0] * rng.uniform(0.9, 1.1), *rng.uniform(-300, 300, 3), base[1] * rng.uniform(0.5, 2.0)]
        for d in range(3):
            assert np.allclose(O.hllc(eos, q, q, d), _phys_flux(eos, q, d), rtol=1e-13, atol=1e-9)


def test_hllc_resolves_an_isolated_contact_exactly():
    # equal p and u, different densities: the flux is the physical flux of the upwind side
    qL = [1.0, 10.0, 3.0, -2.0, 1e5]
    qR = [4.0, 10.0, -1.0, 5.0, 1e5]
    assert np.allclose(O.hllc(AIR, qL, qR, 0), _phys_flux(AIR, qL, 0), rtol=1e-13)
    qL2 = [1.0, -10.0, 3.0, -2.0, 1e5]
    qR2 = [4.0, -10.0, -1.0, 5.0, 1e5]
    assert np.allclose(O.hllc(AIR, qL2, qR2, 0), _phys_flux(AIR, qR2, 0), rtol=1e-13)


def test_hllc_mirror_and_rotation_symmetry():
    rng = np.random.default_rng(2)
    for _ in range(20):
        qL = [1000 * rng.uniform(0.8, 1.2), *rng.uniform(-200, 200, 3), 1e8 * rng.uniform(0.5, 2)]
        qR = [1000 * rng.uniform(0.8, 1.2), *rng.uniform(-200, 200, 3), 1e8 * rng.uniform(0.5, 2)]
        F = O.hllc(WATER, qL, qR, 0)
        # mirror x -> -x: swap sides and negate the normal velocity
        mL = [qR[0], -qR[1], qR[2], qR[3], qR[4]]
        mR = [qL[0], -qL[1], qL[2], qL[3], qL[4]]
        G = O.hllc(WATER, mL, mR, 0)
        assert np.allclose([G[0], G[1], G[2], G[3], G[4]], [-F[0], F[1], -F[2], -F[3], -F[4]], rtol=1e-12,
                           atol=1e-6 * np.abs(F).max())
        # rotation: the y-flux of (u, v, w) -> (w, u, v) equals the x-flux permuted
        rL = [qL[0], qL[3], qL[1], qL[2], qL[4]]
        rR = [qR[0], qR[3], qR[1], qR[2], qR[4]]
        H = O.hllc(WATER, rL, rR, 1)
        assert np.allclose([H[0], H[2], H[3], H[1], H[4]], F, rtol=1e-12, atol=1e-6 * np.abs(F).max())


@pytest.mark.parametrize("eos", [WATER, AIR])
def test_hllc_star_state_energy_satisfies_the_jump_condition(eos):
    """Pins the HLLC star energy (App. C.4; reading R13): when the flux is a star flux
    F*_K = F_K + S_K (U*_K - U_K), the star state recovered from it must carry the contact
    speed S* as its normal velocity, the side's tangential velocities, and an energy whose
    physical flux S* ((rho E)*_K + p*) equals F*'s energy component, with
    p* = p_K + rho_K (S_K - u_K)(S* - u_K) (the jump conditions across S_K). A dropped or
    mis-signed term in E*_K breaks the last identity."""
    rng = np.random.default_rng(21)
    g = eos.prm[0]
    base = (1000.0, 1e8) if eos is WATER else (1.2, 1e5)
    checked = {"L": 0, "R": 0}
    for _ in range(400):
        qL = [base[0] * rng.uniform(0.7, 1.3), *rng.uniform(-150, 150, 3), base[1] * rng.uniform(0.3, 3.0)]
        qR = [base[0] * rng.uniform(0.7, 1.3), *rng.uniform(-150, 150, 3), base[1] * rng.uniform(0.3, 3.0)]
        cL, cR = (math.sqrt(O.sound_speed2(eos, q[0], q[4])) for q in (qL, qR))
        SL, SR = min(qL[1] - cL, qR[1] - cR), max(qL[1] + cL, qR[1] + cR)
        if not (SL < 0.0 < SR):
            continue
        F = O.hllc(eos, qL, qR, 0)
        for side, q, S in (("L", qL, SL), ("R", qR, SR)):
            U = _cons(eos, q)
            Ustar = U + (F - _phys_flux(eos, q, 0)) / S
            Sstar = Ustar[1] / Ustar[0]
            # F is this side's star flux only if 0 lies between S_K and S*
            if not ((side == "L" and Sstar >= 0.0) or (side == "R" and Sstar < 0.0)):
                continue
            pstar = q[4] + q[0] * (S - q[1]) * (Sstar - q[1])
            assert Ustar[2] / Ustar[0] == pytest.approx(q[2], rel=1e-9, abs=1e-6)
            assert Ustar[3] / Ustar[0] == pytest.approx(q[3], rel=1e-9, abs=1e-6)
            assert F[1] == pytest.approx(Ustar[1] * Sstar + pstar, rel=1e-10)
            assert F[4] == pytest.approx(Sstar * (Ustar[4] + pstar), rel=1e-9, abs=1e-9 * abs(U[4] * S))
            checked[side] += 1
    assert checked["L"] > 20 and checked["R"] > 20, checked


def _cons(eos, q):
    rho, u, v, w, p = q
    E = O.energy(eos, rho, p) + 0.5 * (u * u + v * v + w * w)
    return np.array([rho, rho * u, rho * v, rho * w, rho * E])


# --------------------------------------------------------------------------- exact Riemann solver

def _e_sg(eos, rho, p):
    g, pc = eos.prm
    return (p + g * pc) / ((g - 1.0) * rho)


def _rh_residuals(e_fn, ahead, behind):
    """Relative residuals of mass, momentum and energy conservation across a shock between
    ahead = (rho, u, p) and behind = (rho, u, p), shock speed from mass conservation."""
    r0, u0, p0 = ahead
    r1, u1, p1 = behind
    S = (r1 * u1 - r0 * u0) / (r1 - r0)
    m0, m1 = r0 * (u0 - S), r1 * (u1 - S)
    E0 = e_fn(r0, p0) + 0.5 * u0 ** 2
    E1 = e_fn(r1, p1) + 0.5 * u1 ** 2
    mom = (m0 * (u0 - S) + p0) - (m1 * (u1 - S) + p1)
    en = (m0 * (E0 - 0.5 * u0 ** 2 + 0.5 * (u0 - S) ** 2) + p0 * (u0 - S)) - \
         (m1 * (E1 - 0.5 * u1 ** 2 + 0.5 * (u1 - S) ** 2) + p1 * (u1 - S))
    scale_m = abs(m0 * (u0 - S)) + abs(p0) + abs(p1)
    scale_e = abs(m0 * E0) + abs(p0 * (u0 - S)) + abs(p1 * (u1 - S))
    return abs(m0 - m1) / abs(m0), abs(mom) / scale_m, abs(en) / scale_e


def test_shock_tube_star_state_satisfies_jump_conditions_and_invariants():
    """The water | air problem of the 1D shock-tube workload: a water rarefaction and an air shock.
    Shock side: Rankine-Hugoniot conservation. Rarefaction side: isentrope (p + p_c)/rho^gamma
    and Riemann invariant u + 2c/(gamma - 1) constant (stiffened gas)."""
    wL, wR = (1000.0, 0.0, 1e9), (1.0, 0.0, 1e5)
    (ps, us, rl, rr), _ = O.riemann(WATER, wL, AIR, wR)
    assert ps < wL[2] and ps > wR[2]
    for res in _rh_residuals(lambda r, p: _e_sg(AIR, r, p), (wR[0], wR[1], wR[2]), (rr, us, ps)):
        assert res < 1e-12
    g, pc = WATER.prm
    assert (ps + pc) / rl ** g == pytest.approx((wL[2] + pc) / wL[0] ** g, rel=1e-12)
    cL = math.sqrt(g * (wL[2] + pc) / wL[0])
    cs = math.sqrt(g * (ps + pc) / rl)
    assert us + 2 * cs / (g - 1) == pytest.approx(wL[1] + 2 * cL / (g - 1), rel=1e-12)


def _brute_force_sg(eosL, wL, eosR, wR):
    """Independent solution of a two-stiffened-gas Riemann problem: shock branches from the
    Rankine-Hugoniot relations solved numerically, rarefaction branches by integrating
    du = -dp/(rho c) along the isentrope with scipy, and the star pressure by brentq."""
    from scipy.optimize import brentq

    def side(eos, w, p, sgn):
        g, pc = eos.prm
        rho0, u0, p0 = w
        if p > p0:
            # density behind the shock from the Hugoniot energy equation
            def H(r):
                return _e_sg(eos, r, p) - _e_sg(eos, rho0, p0) - 0.5 * (p + p0) * (1 / rho0 - 1 / r)
            r = brentq(H, rho0 * (1 + 1e-15), rho0 * (g + 1) / (g - 1) * (1 - 1e-12), xtol=1e-300, rtol=1e-15)
            du = math.sqrt((p - p0) * (1 / rho0 - 1 / r))
            return u0 - sgn * du, r
        sol = solve_ivp(lambda q, y: [y[0] / (g * (q + pc)), 1.0 / math.sqrt(g * (q + pc) * y[0])],
                        (p0, p), [rho0, 0.0], rtol=1e-13, atol=1e-14, method="DOP853")
        r, f = sol.y[0, -1], sol.y[1, -1]
        return u0 - sgn * f, r

    def F(p):
        return side(eosL, wL, p, 1)[0] - side(eosR, wR, p, -1)[0]

    lo = max(-eosL.prm[1], -eosR.prm[1]) * (1 - 1e-12) + 1e-9
    ps = brentq(F, lo, 1e11, xtol=1e-300, rtol=1e-15)
    uL, rl = side(eosL, wL, ps, 1)
    uR, rr = side(eosR, wR, ps, -1)
    return ps, 0.5 * (uL + uR), rl, rr


@pytest.mark.parametrize("wL,wR,eosL,eosR", [
    ((1000.0, 0.0, 1e9), (1.0, 0.0, 1e5), WATER, AIR),       # shock-tube workload
    ((1.2, 0.0, 1e5), (1000.0, 0.0, 1e9), AIR, WATER),       # mirrored roles
    ((1000.0, 300.0, 1e5), (1.2, -100.0, 1e5), WATER, AIR),  # collision: two shocks
    ((1000.0, -50.0, 1e6), (1.2, 200.0, 1e5), WATER, AIR),   # expansion: two rarefactions
])
def test_riemann_matches_brute_force(wL, wR, eosL, eosR):
    (ps, us, rl, rr), _ = O.riemann(eosL, wL, eosR, wR)
    bp, bu, brl, brr = _brute_force_sg(eosL, wL, eosR, wR)
    assert ps == pytest.approx(bp, rel=1e-9)
    assert us == pytest.approx(bu, rel=1e-9, abs=1e-9 * (abs(wL[1]) + abs(wR[1]) + 1.0))
    assert rl == pytest.approx(brl, rel=1e-9)
    assert rr == pytest.approx(brr, rel=1e-9)


def _sg_curve(g, pc, rho, p, ps):
    """Textbook stiffened-gas wave curve f_K(p*) in P = p + p_c (shock: Rankine-Hugoniot;
    rarefaction: the isentrope), written here independently of the oracle."""
    P, PK = ps + pc, p + pc
    if ps >= p:
        A, B = 2.0 / ((g + 1.0) * rho), (g - 1.0) / (g + 1.0) * PK
        return (ps - p) * math.sqrt(A / (P + B))
    c = math.sqrt(g * PK / rho)
    return 2.0 * c / (g - 1.0) * ((P / PK) ** ((g - 1.0) / (2.0 * g)) - 1.0)


@pytest.mark.parametrize("wL,wR,eosL,eosR", [
    ((1000.0, 0.0, 1e9), (1.2, 0.0, 1e5), WATER, AIR),
    ((1000.0, 300.0, 1e5), (1.2, -100.0, 1e5), WATER, AIR),
    ((1000.0, -50.0, 1e6), (1.2, 200.0, 1e5), WATER, AIR),
    ((1.0, 0.0, 1e5), (0.125, 0.0, 1e4), AIR, AIR),
    ((1000.0, 5.0, 2e8), (1000.0, -5.0, 1e8), WATER, WATER),
])
def test_riemann_star_pressure_to_the_newton_tolerance(wL, wR, eosL, eosR):
    """Reading R6 stops the Newton iteration at the first step with |dp| <= 1e-12 |p| and keeps
    that step's update: on closed-form stiffened-gas curves the oracle's p* then agrees with the
    root of the same F(p) = f_L + f_R + u_R - u_L, found by bracketing to 1e-15, within 1e-14
    (the rounding level of F). A tolerance of 1e-6, or a stop before the last update, fails it
    (both checked by planting them in the oracle)."""
    from scipy.optimize import brentq
    gL, pcL = eosL.prm[0], eosL.prm[1]
    gR, pcR = eosR.prm[0], eosR.prm[1]

    def F(ps):
        return _sg_curve(gL, pcL, wL[0], wL[2], ps) + _sg_curve(gR, pcR, wR[0], wR[2], ps) + (wR[1] - wL[1])
    lo = max(-pcL, -pcR) + 1e-9 * max(wL[2], wR[2])
    root = brentq(F, lo, 1e12, xtol=1e-300, rtol=1e-15)
    (ps, us, rl, rr), _ = O.riemann(eosL, wL, eosR, wR)
    assert ps == pytest.approx(root, rel=1e-14)


@pytest.mark.parametrize("w,p", [((1000.0, 0.0, 1e5), 1e8), ((1000.0, 0.0, 1e5), 2e9), ((1100.0, 50.0, 3e8), 5e9),
                                 ((1000.0, 0.0, 1e5), 1.0001e5)])
def test_mg_shock_density_to_the_hugoniot_tolerance(w, p):
    """The MG shock branch's density solves the Hugoniot energy equation
    H(rho) = e(rho, p) - e_K - (p + p_K)(1/rho_K - 1/rho)/2 = 0 (Sec. 4.2, App. B.3), found by
    Newton stopped at the first step below 1e-14 rho (Reading R6): within 1e-14 of the root found
    by bracketing the same H (with the oracle's e(rho, p), pinned above). A Newton tolerance of
    1e-7 planted in the oracle fails it."""
    from scipy.optimize import brentq
    eK = O.energy(MGW, w[0], w[2])

    def H(r):
        return O.energy(MGW, r, p) - eK - 0.5 * (p + w[2]) * (1.0 / w[0] - 1.0 / r)
    hi = 1000.0 * 1.75 / 0.75 * (1.0 - 1e-12)
    root = brentq(H, w[0] * (1.0 + 1e-15), hi, xtol=1e-300, rtol=1e-15)
    _, _, rho = O.wave_curve(MGW, w, p)
    assert rho == pytest.approx(root, rel=1e-14)


def test_riemann_trivial_and_symmetric_cases():
    w = (1000.0, 12.0, 3e7)
    (ps, us, rl, rr), _ = O.riemann(WATER, w, WATER, w)
    assert (ps, us, rl, rr) == (w[2], w[1], w[0], w[0])
    (ps, us, rl, rr), _ = O.riemann(MGW, (1000.0, 0.0, 1e5), MGW, (1000.0, 0.0, 1e5))
    assert (ps, us) == (1e5, 0.0) and rl == rr == 1000.0
    # symmetric collision: u* = 0 and equal star densities
    (ps, us, rl, rr), _ = O.riemann(MGW, (1000.0, 250.0, 1e5), MGW, (1000.0, -250.0, 1e5))
    assert abs(us) < 1e-9 and rl == pytest.approx(rr, rel=1e-13)
    # mirror: swap the sides and negate the velocities
    a, _ = O.riemann(WATER, (1000.0, 30.0, 2e8), AIR, (1.2, -5.0, 1e5))
    b, _ = O.riemann(AIR, (1.2, 5.0, 1e5), WATER, (1000.0, -30.0, 2e8))
    assert a[0] == pytest.approx(b[0], rel=1e-12)
    assert a[1] == pytest.approx(-b[1], rel=1e-12)
    assert a[2] == pytest.approx(b[3], rel=1e-12) and a[3] == pytest.approx(b[2], rel=1e-12)


def test_riemann_vacuum_is_reported():
    assert O.riemann_status(AIR, (1.0, -2e4, 1e5), AIR, (1.0, 2e4, 1e5)) == 6  # EVACUUM


def test_paper_test12_glass_side_density():
    """Sec. 5.1, Test 12: air | soda-lime glass (MG), glass moving away at 1500 m/s. The paper
    prints the glass-side density next to the interface as 2203.98 kg/m^3."""
    with open(os.path.join(HERE, "golden", "test12_riemann.json")) as f:
        g = json.load(f)
    L, R = g["left"], g["right"]
    prmR = [float(x) for x in R["prm"]]
    (ps, us, rl, rr), _ = O.riemann(O.EOS(O.EOS_SG, tuple(L["prm"])), (L["rho"], L["u"], L["p"]),
                                    O.EOS(O.EOS_MG, tuple(prmR)), (R["rho"], R["u"], R["p"]))
    assert abs(rr - g["rho_star_right"]) <= g["rho_star_right_abs_tol"]
    assert 0.0 < ps < 1e5 and rl < 1.2   # both waves are rarefactions (Sec. 5.1)


def test_mg_shock_from_reference_state_follows_linear_us_up():
    """The MG compression curve p_R(eta) = rho0 c0^2 eta/(1 - s eta)^2 with e_R = p_R eta/(2 rho0) + e0
    is the Hugoniot of a material with the linear shock law U_s = c0 + s u_p, centred on the
    reference state (rho0, p = 0, e0). A shock from that state must follow it."""
    for p1 in (1e7, 1e8, 1e9, 5e9):
        rho1, u1, S = O.shock_state(MGW, (1000.0, 0.0, 0.0), p1)
        assert S == pytest.approx(1483.0 + 1.75 * u1, rel=1e-11)
        eta = 1.0 - 1000.0 / rho1
        assert p1 == pytest.approx(1000.0 * 1483.0 ** 2 * eta / (1 - 1.75 * eta) ** 2, rel=1e-11)


@pytest.mark.parametrize("eos,w,p1", [(MGW, (1000.0, 0.0, 1e5), 1e9), (MGW, (1100.0, 50.0, 2e8), 3e9),
                                      (WATER, (1000.0, 0.0, 1e5), 1e9)])
def test_shock_state_satisfies_rankine_hugoniot(eos, w, p1):
    rho1, u1, S = O.shock_state(eos, w, p1)
    for res in _rh_residuals(lambda r, p: O.energy(eos, r, p), w, (rho1, u1, p1)):
        assert res < 1e-11


@pytest.mark.parametrize("w,p,tol", [((1000.0, 0.0, 1e9), 1e5, 1e-8), ((1000.0, 0.0, 1e5), -5e6, 1e-8),
                                     ((1250.0, 0.0, 2e9), 1.5e9, 1e-8), ((2204.0, 0.0, 1e5), 0.03, 1e-8),
                                     ((1250.0, 0.0, 2e9), 3e8, 2e-5)])
def test_mg_rarefaction_matches_ode_integration(w, p, tol):
    """The RK4 isentrope of the MG rarefaction against scipy's DOP853 on the energy form
    de/drho = p/rho^2 (first law at constant entropy), c^2 pinned by the identity test above.
    The last case crosses eta = 0, where c^2 has a kink, so 64 RK4 substeps are only
    accurate to a few 1e-6 there."""
    eos = MGW if w[0] < 2000 else O.EOS(O.EOS_MG, (2204.0, 2220.0, 1.61, 0.65, 0.0, -math.inf))
    f, df, rho_star = O.wave_curve(eos, w, p)
    e0 = O.energy(eos, w[0], w[2])

    def rhs(r, y):
        e, fv = y
        pr = O.pressure(eos, r, e)
        return [pr / r ** 2, math.sqrt(O.sound_speed2(eos, r, pr)) / r]

    def hit(r, y):
        return O.pressure(eos, r, y[0]) - p
    hit.terminal = True
    sol = solve_ivp(rhs, (w[0], 0.5 * w[0]), [e0, 0.0], events=hit, rtol=1e-11, atol=1e-12, method="DOP853")
    r_end = sol.t_events[0][0]
    f_end = sol.y_events[0][0][1]
    assert rho_star == pytest.approx(r_end, rel=tol)
    assert f == pytest.approx(f_end, rel=max(tol, 1e-7), abs=1e-9)
    # derivative of the wave curve is 1/(rho c) at the end state (Sec. 4.2, isentrope)
    assert df == pytest.approx(1.0 / (rho_star * math.sqrt(O.sound_speed2(eos, rho_star, p))), rel=1e-12)


# --------------------------------------------------------------------------- flow solver

def _grid(setup, **kw):
    return O.Grid(n=setup.n, h=setup.h, eos=tuple(O.EOS(*e) for e in setup.eos), bc=setup.bc,
                  cfl=setup.cfl, reinit_every=kw.get("reinit_every", setup.reinit_every),
                  reinit_iters=setup.reinit_iters)


def _periodic_setup(n, seed, two_phase=False):
    P, phi = WL.random_state(n, seed, two_phase=two_phase)
    s = WL.Setup("random", n, 1.0 / n[0], (WL.WATER_SG, WL.AIR_PG), (1,) * 6, phi,
                 np.zeros(phi.shape, np.uint8), {})
    return s, P


def test_time_step_closed_form():
    s, P = _periodic_setup((8, 8, 8), 0)
    P[...] = np.array([1000.0, 10.0, -20.0, 5.0, 1e8])[:, None, None, None]
    g = _grid(s)
    W = O.prims_to_cons(g, P, s.phi)
    c = math.sqrt(6.12 * (1e8 + 3.43e8) / 1000.0)
    assert O.time_step(g, W, s.phi) == pytest.approx(0.5 * s.h / (35.0 + 3 * c), rel=1e-14)


def test_uniform_flow_is_preserved_bitwise():
    s, P = _periodic_setup((8, 6, 5), 0)
    P[...] = np.array([1000.0, 10.0, -20.0, 5.0, 1e8])[:, None, None, None]
    g = _grid(s)
    W = O.prims_to_cons(g, P, s.phi)
    r = O.run(g, W, s.phi, 5)
    for v in range(5):
        assert np.all(r.W[v] == W[v][0, 0, 0])


def test_single_material_periodic_run_conserves_mass_momentum_energy():
    s, P = _periodic_setup((12, 10, 8), 5)
    g = _grid(s)
    W = O.prims_to_cons(g, P, s.phi)
    r = O.run(g, W, s.phi, 20)
    for v in range(5):
        tot0 = W[v].sum()
        scale = np.abs(W[v]).sum()
        assert abs(r.W[v].sum() - tot0) <= 1e-13 * scale
    assert not np.allclose(r.W[0], W[0])   # the state did evolve


def test_two_material_contact_at_rest_stays_at_rest():
    s, P = _periodic_setup((10, 8, 8), 1, two_phase=True)
    P[0] = np.where(s.phi < 0, 1.2, 1000.0)
    P[1:4] = 0.0
    P[4] = 1e5
    g = _grid(s)
    W = O.prims_to_cons(g, P, s.phi)
    r = O.run(g, W, s.phi, 3)
    assert np.array_equal(r.W, W)


def test_shock_bubble_is_mirror_symmetric():
    s = WL.shock_bubble(n=24, radius=0.2, steps=30)
    g = _grid(s)
    rho1, u1, _ = O.shock_state(O.EOS(*s.eos[0]), (1000.0, 0.0, 1e5), 1e9)
    W = O.prims_to_cons(g, s.prims((rho1, u1)), s.phi)
    r = O.run(g, W, s.phi, 30)
    assert r.stats["interface_faces"] > 0
    for v in range(5):
        a = r.W[v]
        scale = np.abs(a).max()
        sgn_y = -1.0 if v == 2 else 1.0
        sgn_z = -1.0 if v == 3 else 1.0
        assert np.abs(a - sgn_y * a[:, ::-1, :]).max() <= 1e-12 * scale
        assert np.abs(a - sgn_z * a[::-1, :, :]).max() <= 1e-12 * scale
    # y <-> z exchange swaps the v and w momenta
    sw = {2: 3, 3: 2}
    for v in range(5):
        b = r.W[sw.get(v, v)].transpose(1, 0, 2)
        assert np.abs(r.W[v] - b).max() <= 1e-12 * np.abs(r.W[v]).max()
    assert np.array_equal(r.phi < 0, (r.phi < 0)[:, ::-1, :])


def test_shock_tube_converges_to_exact_solution():
    """Water | air shock tube on nx x 1 x 1 grids: L1 error of density against the exact
    two-stiffened-gas solution decreases under refinement (Sec. 5.1 verification approach)."""
    errs = []
    for nx in (64, 128, 256, 512):
        s = WL.shock_tube(nx=nx, ny=1, nz=1)
        g = _grid(s)
        W = O.prims_to_cons(g, s.prims(), s.phi)
        r = O.run(g, W, s.phi, nx // 2)
        P = O.cons_to_prims(g, r.W, r.phi)
        x = (np.arange(nx) + 0.5) / nx
        ex, _ = O.exact_sample_sg(WATER.prm, (1000.0, 0.0, 1e9), AIR.prm, (1.0, 0.0, 1e5), (x - 0.5) / r.t)
        errs.append(np.abs(P[0, 0, 0] - ex[0]).mean() / np.abs(ex[0]).mean())
        # interface position: the sign change of phi sits within two cells of x = 0.5 + u* t
        _, star = O.exact_sample_sg(WATER.prm, (1000.0, 0.0, 1e9), AIR.prm, (1.0, 0.0, 1e5), np.zeros(1))
        xi = x[np.argmax(r.phi[0, 0] >= 0.0)]
        assert abs(xi - (0.5 + star[1] * r.t)) <= 2.0 / nx
    assert all(b < a for a, b in zip(errs, errs[1:]))
    order = math.log(errs[0] / errs[-1], 2) / 3
    assert order > 0.5


def test_smooth_entropy_wave_converges_at_second_order():
    """A density sine wave carried by uniform velocity and pressure (perfect gas, periodic in x)
    is translated exactly by the Euler equations, and so is a smooth level set by u phi_x. MUSCL
    with the smooth van Albada slope, HLLC and the RK2 average (Sec. 4.1, App. D) are second order
    there: the L1 errors of rho and phi against the translated profiles fall by about 4 per
    halving of h. Dropping the RK2 average of W or the half of the slope in the face states
    makes the rho order about 1; dropping the RK2 average of phi makes the phi order about 1."""
    air = O.EOS(O.EOS_SG, (1.4, 0.0))
    u, T = 1.0, 0.5
    err_rho, err_phi = [], []
    for nx in (32, 64, 128, 256):
        h = 1.0 / nx
        g = O.Grid(n=(nx, 1, 1), h=h, eos=(air, air), bc=(1, 1, 0, 0, 0, 0), reinit_every=10 ** 9)
        x = (np.arange(nx) + 0.5) * h
        P = np.zeros((5, 1, 1, nx))
        P[0, 0, 0] = 1.0 + 0.2 * np.sin(2 * np.pi * x)
        P[1] = u
        P[4] = 1.0
        phi = (0.5 + 0.3 * np.sin(2 * np.pi * x))[None, None, :]   # positive: one material
        W = O.prims_to_cons(g, P, phi)
        n = int(math.ceil(T / O.time_step(g, W, phi)))
        r = O.run(g, W, phi, n)
        assert r.stats["interface_faces"] == 0
        Pn = O.cons_to_prims(g, r.W, r.phi)
        xs = x - u * r.t
        err_rho.append(np.abs(Pn[0, 0, 0] - (1.0 + 0.2 * np.sin(2 * np.pi * xs))).mean())
        err_phi.append(np.abs(r.phi[0, 0] - (0.5 + 0.3 * np.sin(2 * np.pi * xs))).mean())
    for errs in (err_rho, err_phi):
        orders = [math.log2(a / b) for a, b in zip(errs, errs[1:])]
        assert min(orders) > 1.7, orders
        assert math.log2(errs[0] / errs[-1]) / 3 > 1.85, orders


def test_level_set_stencil_is_exact_for_cubics():
    """The third-order upwind-biased derivative (Sec. 4.4) differentiates cubic polynomials
    exactly, so the level-set residual of phi = cubic(x) in a uniform flow is -u phi'(x)."""
    n = (16, 4, 4)
    s, P = _periodic_setup(n, 0)
    s = WL.Setup("lin", n, 1.0 / 16, (WL.WATER_SG, WL.AIR_PG), (0,) * 6, s.phi, s.region, {})
    x, y, z = WL.cell_centres(n, s.h)
    for u in (37.0, -23.0):
        P[...] = np.array([1000.0, u, 0.0, 0.0, 1e8])[:, None, None, None]
        phi = 0.3 + 0.5 * (x - 0.4) - 2.0 * (x - 0.4) ** 2 + 1.5 * (x - 0.4) ** 3
        g = _grid(s)
        W = O.prims_to_cons(g, P, np.abs(phi) + 1.0)
        R, L, _ = O.residual(g, W, phi)
        dphi = 0.5 - 4.0 * (x - 0.4) + 4.5 * (x - 0.4) ** 2
        inner = slice(2, -2)
        assert np.allclose(L[:, :, inner], (-u * dphi)[:, :, inner], rtol=1e-11, atol=1e-9)


def test_reinit_keeps_a_plane_distance_and_every_sign():
    n = (20, 6, 6)
    g = O.Grid(n=n, h=1.0 / 20, eos=(O.EOS(*WL.WATER_SG), O.EOS(*WL.AIR_PG)), bc=(0,) * 6)
    x, y, z = WL.cell_centres(n, 1.0 / 20)
    phi = x - 0.43
    out = O.reinit(g, phi, 5)
    assert np.abs(out - phi)[:, :, 1:-1].max() < 1e-12
    # a rough level set keeps every sign (first layer frozen, Sec. 4.4)
    rng = np.random.default_rng(3)
    phi2 = (x - 0.5) * rng.uniform(0.2, 3.0, size=x.shape)
    out2 = O.reinit(g, phi2, 10)
    assert np.array_equal(out2 < 0, phi2 < 0)
    # a steep plane relaxes to the signed distance, |grad phi| = 1 (Eq. signed_distance_property)
    phi3 = 2.5 * (x - 0.5)
    out3 = O.reinit(g, phi3, 60)
    grad = np.diff(out3, axis=2) / (1.0 / 20)
    away = np.ones(grad.shape[2], bool)
    away[[0, 1, 9, grad.shape[2] - 2, grad.shape[2] - 1]] = False   # boundary faces and the frozen pair
    assert np.abs(grad[:, :, away] - 1.0).max() < 1e-6
    assert np.array_equal(out3 < 0, phi3 < 0)


def test_phase_update_follows_translating_interface():
    """Uniform flow u = 100 m/s carrying an air | water plane interface: every cell that changes
    material gets a state of its new material, and the interface moves by u t to within a cell."""
    nx = 64
    s = WL.shock_tube(nx=nx, ny=1, nz=1)
    P = s.prims()
    P[1] = 100.0
    P[4] = 1e5
    g = _grid(s)
    W = O.prims_to_cons(g, P, s.phi)
    r = O.run(g, W, s.phi, 60)
    Q = O.cons_to_prims(g, r.W, r.phi)
    water = r.phi < 0
    assert np.all(np.abs(Q[0][water] - 1000.0) < 1.0) and np.all(np.abs(Q[0][~water] - 1.0) < 0.01)
    x = (np.arange(nx) + 0.5) / nx
    xi = x[np.argmax(r.phi[0, 0] >= 0.0)]
    assert abs(xi - (0.5 + 100.0 * r.t)) <= 1.0 / nx
    assert r.stats["flipped"] > 0


def _undershoot_setup():
    """A 1D periodic water column in slow uniform flow whose level set has a small positive
    value next to a steep profile, so that the third-order stencil drives that one cell
    negative while every neighbour stays positive: a would-be air cell with no air around."""
    n = (16, 1, 1)
    phi = np.full((1, 1, 16), 10.0)
    phi[0, 0, 6] = 0.1
    phi[0, 0, 7] = 0.01
    P = np.zeros((5, 1, 1, 16))
    P[0] = 1000.0
    P[1] = 20.0
    P[4] = 1e8
    s = WL.Setup("undershoot", n, 1.0 / 16, (WL.WATER_SG, WL.AIR_PG), (1,) * 6, phi,
                 np.zeros(phi.shape, np.uint8), {}, reinit_every=0)
    return s, P


def test_isolated_flip_keeps_its_material():
    s, P = _undershoot_setup()
    g = _grid(s, reinit_every=0)
    W = O.prims_to_cons(g, P, s.phi)
    R, L, _ = O.residual(g, W, s.phi)
    assert L[0, 0, 7] * O.time_step(g, W, s.phi) < -0.01   # the level set alone would go negative
    r = O.run(g, W, s.phi, 1)
    assert r.stats["flipped"] == 1
    assert np.all(r.phi >= 0.0)                              # no sub-cell air fragment is created
    assert np.allclose(r.W, W, rtol=1e-14)                   # uniform water state untouched


def test_reinit_holds_the_first_layer_and_moves_the_rest():
    """Reading R25 (the fixed first layer of Sec. 4.4): cells with a face neighbour of the other
    sign keep their values bit for bit, so the zero level set between them stays where it was,
    while the other cells of a level set that is not a distance move towards one."""
    n = (20, 8, 8)
    h = 1.0 / 20
    g = O.Grid(n=n, h=h, eos=(O.EOS(*WL.WATER_SG), O.EOS(*WL.AIR_PG)), bc=(0,) * 6)
    x, y, z = WL.cell_centres(n, h)
    r = np.sqrt((x - 0.5) ** 2 + (y - 0.2) ** 2 + (z - 0.2) ** 2)
    phi = (r - 0.3) * (1.0 + 2.0 * (x - 0.5) ** 2 + y)        # same zero set as r - 0.3, not a distance
    neg = phi < 0
    first = np.zeros(phi.shape, bool)
    for ax in range(3):
        for sh in (1, -1):
            nb = np.roll(neg, sh, axis=ax)
            edge = [slice(None)] * 3
            edge[ax] = 0 if sh == 1 else -1                      # transmissive: the clamped neighbour is itself
            nb[tuple(edge)] = neg[tuple(edge)]
            first |= nb != neg
    out = O.reinit(g, phi, 8)
    assert first.any() and (~first).any()
    assert np.array_equal(out[first], phi[first])
    assert np.array_equal(out < 0, neg)
    moved = np.abs(out - phi)[~first]
    assert moved.max() > 0.1 * h
    # the moved cells come closer to the distance to the sphere
    dist = r - 0.3
    far = ~first & (np.abs(dist) < 0.25)
    assert np.abs(out - dist)[far].mean() < 0.5 * np.abs(phi - dist)[far].mean()


def test_phase_update_takes_face_neighbours_before_the_26_neighbourhood():
    """Reading R17: a cell that changes material takes the mean primitive state of its face
    neighbours that were and are of the new material; only without any such face neighbour the
    mean over the 26-neighbourhood's; then its conserved state from the new material's EOS."""
    n = (5, 5, 5)
    water, air = O.EOS(*WL.WATER_SG), O.EOS(*WL.AIR_PG)
    g = O.Grid(n=n, h=0.1, eos=(water, air), bc=(0,) * 6)
    shape = (5, 5, 5)

    def case(face_air):
        P = np.zeros((5,) + shape)
        P[0], P[4] = 1000.0, 1e6
        phi = np.ones(shape)
        # air neighbours of the centre (2, 2, 2) [z, y, x]: face ones with states A, an edge one with B
        A = {(2, 2, 1): (1.1, 3.0, 0.0, 0.0, 2e5), (2, 2, 3): (1.3, 5.0, 0.0, 0.0, 4e5)}
        B = {(2, 3, 3): (2.0, -40.0, 7.0, 0.0, 9e5)}
        cells = {**(A if face_air else {}), **B}
        for c, q in cells.items():
            P[(slice(None),) + c] = q
            phi[c] = -1.0
        id_old = (phi < 0).astype(np.uint8)
        W = O.prims_to_cons(g, P, phi)
        phi[2, 2, 2] = -0.5                      # the centre changes from water to air
        W2, phi2, nf = O.phase_fix(g, W, phi, id_old)
        assert nf == 1 and phi2[2, 2, 2] < 0
        got = O.cons_to_prims(g, W2, phi2)[(slice(None), 2, 2, 2)]
        src = A if face_air else B
        want = np.mean(np.array(list(src.values())), axis=0)
        assert np.allclose(got, want, rtol=1e-12, atol=1e-9)
        untouched = np.ones(shape, bool)
        untouched[2, 2, 2] = False
        assert np.array_equal(W2[:, untouched], W[:, untouched])

    case(face_air=True)    # face neighbours A present: the edge neighbour B is ignored
    case(face_air=False)   # no face neighbour of the new material: the 26-neighbourhood (B)


def test_muscl_stencil_stops_at_the_interface():
    """Reading R11: along an axis where a stencil neighbour has the other material the face
    states are first order. So the residual of a cell two cells from the interface does not see
    the state across it (its neighbour's face state towards it is that neighbour's cell state),
    while the cell next to the interface does (through FIVER)."""
    n = (8, 1, 1)
    water, air = O.EOS(*WL.WATER_SG), O.EOS(*WL.AIR_PG)
    g = O.Grid(n=n, h=0.1, eos=(water, air), bc=(0,) * 6)
    x = (np.arange(8) + 0.5) * 0.1
    phi = (0.4 - x)[None, None, :]                 # cells 0-3 water (phi > 0), 4-7 air
    P = np.zeros((5, 1, 1, 8))
    P[0] = np.where(phi < 0, 1.2, 1000.0) * (1 + 0.05 * np.sin(7 * x))
    P[1] = 3.0 * np.cos(5 * x)
    P[4] = np.where(phi < 0, 1e5, 2e5) * (1 + 0.1 * x)
    W = O.prims_to_cons(g, P, phi)
    R0, _, _ = O.residual(g, W, phi)
    P2 = P.copy()
    P2[0, 0, 0, 4] *= 1.7                          # the first air cell: denser, higher pressure
    P2[4, 0, 0, 4] *= 3.0
    W2 = O.prims_to_cons(g, P2, phi)
    R2, _, _ = O.residual(g, W2, phi)
    assert np.array_equal(R2[:, 0, 0, 2], R0[:, 0, 0, 2])
    assert not np.allclose(R2[:, 0, 0, 3], R0[:, 0, 0, 3])


def test_zero_level_set_belongs_to_material_zero():
    """The material of a cell is 1 where phi < 0 and 0 elsewhere, phi = 0 and phi = -0.0
    included. Water under tension (p = -1e7 Pa, admissible for the stiffened gas with
    p_c = 3.43e8) on cells with phi = +-0 stays water: a uniform state is kept bit for bit
    (as air the state would be non-physical)."""
    n = (6, 1, 1)
    g = O.Grid(n=n, h=0.1, eos=(O.EOS(*WL.WATER_SG), O.EOS(*WL.AIR_PG)), bc=(1,) * 6)
    phi = np.array([1.0, 0.5, 0.0, -0.0, 0.5, 1.0])[None, None, :]
    P = np.zeros((5, 1, 1, 6))
    P[0] = 1000.0
    P[4] = -1e7
    W = O.prims_to_cons(g, P, phi)
    r = O.run(g, W, phi, 3)
    assert np.array_equal(r.W, W)
    assert r.stats["interface_faces"] == 0
