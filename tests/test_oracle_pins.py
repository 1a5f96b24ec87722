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


def test_a_state_without_sound_speed_is_not_admissible():
    """c^2 > 0 is required of every state (the wave speeds u -+ c of App. C.4 and the 1/(rho c)
    of the wave curves, Sec. 4.2): a stiffened gas at p = -p_c has c = 0 and is rejected, as is
    one below it; one just above it is admitted."""
    g, pc = WATER.prm
    for p in (-pc, -pc * (1.0 + 1e-12)):
        with pytest.raises(O.OracleError):
            O.sound_speed2(WATER, 1000.0, p)
    assert O.sound_speed2(WATER, 1000.0, -pc * (1.0 - 1e-9)) > 0.0


def test_primitive_conversion_rejects_a_state_without_sound_speed():
    """The conserved -> primitive conversion of a cell (the first step of each stage) rejects a
    stiffened-gas state whose internal energy puts its pressure below -p_c (no real sound
    speed), reporting the cell, rather than passing it on."""
    g = O.Grid(n=(4, 1, 1), h=0.25, eos=(WATER, AIR), bc=(0,) * 6)
    P = np.zeros((5, 1, 1, 4))
    P[0], P[4] = 1000.0, 1e5
    phi = np.ones((1, 1, 4))
    W = O.prims_to_cons(g, P, phi)
    gam, pc = WATER.prm
    e_bad = (-1.5 * pc + gam * pc) / ((gam - 1.0) * 1000.0)   # p = -1.5 p_c
    W[4, 0, 0, 2] = 1000.0 * e_bad
    with pytest.raises(O.OracleError):
        O.cons_to_prims(g, W, phi)
    code, cell = O.run_status(g, W, phi, 1)
    assert code == 5 and cell == 2    # ENONPHYS at that cell


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
    # two strong water rarefactions whose Newton iteration does not converge within its 50
    # steps: p* comes from the bracketing bisection of Reading R6 (stopped at a bracket of
    # 1e-14 of its ends)
    ((956.875186, -1351.01462, 6.87618598e7), (1211.34497, -1272.28087, 5.27972620e7), WATER, WATER),
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
    (ps, us, rl, rr), iters = O.riemann(eosL, wL, eosR, wR)
    assert ps == pytest.approx(root, rel=1e-14)
    assert (iters > 50) == (wL[1] < -1000.0)   # only the last case reaches the bisection


@pytest.mark.parametrize("w,p", [((1000.0, 0.0, 1e5), 1e8), ((1000.0, 0.0, 1e5), 2e9), ((1100.0, 50.0, 3e8), 5e9),
                                 ((1000.0, 0.0, 1e5), 1.0001e5), ((1000.0, 0.0, 1e5), 3e11)])
def test_mg_shock_density_to_the_hugoniot_tolerance(w, p):
    """The MG shock branch's density solves the Hugoniot energy equation
    H(rho) = e(rho, p) - e_K - (p + p_K)(1/rho_K - 1/rho)/2 = 0 (Sec. 4.2, App. B.3), found by
    Newton stopped at the first step below 1e-14 rho (Reading R6): within 1e-14 of the root found
    by bracketing the same H (with the oracle's e(rho, p), pinned above). A Newton tolerance of
    1e-7 planted in the oracle fails it. The last case (3e11 Pa, rho* above 0.9 of the maximum
    compression rho0 s/(s - 1)) fails a bracket that stops short of that limit."""
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


@pytest.mark.parametrize("eos", [MGW, WATER, AIR])
def test_shock_speed_is_galilean_and_carries_the_momentum_jump(eos):
    """The shock speed returned with a post-shock state: moving the state ahead by a velocity
    moves the shock and the state behind by the same velocity (Galilean invariance of the Euler
    equations), and the speed carries the momentum jump rho0 (u0 - S)^2 + p0 =
    rho1 (u1 - S)^2 + p1 (Rankine-Hugoniot)."""
    w0 = (1000.0, 0.0, 1e5) if eos is not AIR else (1.2, 0.0, 1e5)
    p1 = 1e9 if eos is not AIR else 5e5
    rho_a, u_a, S_a = O.shock_state(eos, w0, p1)
    for du in (75.0, -140.0):
        rho_b, u_b, S_b = O.shock_state(eos, (w0[0], w0[1] + du, w0[2]), p1)
        assert rho_b == pytest.approx(rho_a, rel=1e-13)
        assert u_b == pytest.approx(u_a + du, rel=1e-12)
        assert S_b == pytest.approx(S_a + du, rel=1e-12)
        lhs = w0[0] * (w0[1] + du - S_b) ** 2 + w0[2]
        rhs = rho_b * (u_b - S_b) ** 2 + p1
        assert lhs == pytest.approx(rhs, rel=1e-11)


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


def _isentrope_until(eos, w, stop):
    """Integrates the isentrope through w = (rho, u, p) towards lower density with scipy's DOP853
    on the energy form de/drho = p/rho^2, df/drho = c/rho (f = the velocity change, negative
    below rho_K) until stop(rho, e, f) = 0; returns (rho, p, f) there."""
    e0 = O.energy(eos, w[0], w[2])

    def rhs(r, y):
        pr = O.pressure(eos, r, y[0])
        return [pr / r ** 2, math.sqrt(O.sound_speed2(eos, r, pr)) / r]

    def ev(r, y):
        return stop(r, y[0], y[1])
    ev.terminal = True
    sol = solve_ivp(rhs, (w[0], 0.5 * w[0]), [e0, 0.0], events=ev, rtol=1e-12, atol=1e-12, method="DOP853")
    r = sol.t_events[0][0]
    e, f = sol.y_events[0][0]
    return r, O.pressure(eos, r, e), f


@pytest.mark.parametrize("eos,w,u", [
    (MGW, (1300.0, 0.0, 1e9), 100.0),       # strong rarefactions on the fixed RK4 nodes
    (MGW, (1300.0, 0.0, 2e9), 400.0),
    (MGW, (1000.0, 0.0, 1e5), 20.0),        # into tension, no cutoff
    (MGW_CUT, (1000.0, 0.0, 1e5), 30.0),    # into tension above the cutoff p_min = K0 eta_min
    (MGW_CUT, (1000.0, 0.0, 1e5), 70.0),
])
def test_mg_riemann_rarefactions_match_ode_integration(eos, w, u):
    """Two MG states separating at +-u (Sec. 4.2): by symmetry u* = 0 and p* is where the
    rarefaction's velocity change reaches -u, found here by integrating the isentrope with
    DOP853 (the energy form, c^2 pinned above). This exercises the exact solver's rarefaction
    curves on the problem's fixed RK4 nodes (Reading R6) far from the side state, and, with a
    tensile cutoff, a star pressure below zero but above the cutoff's p_min = rho0 c0^2 eta_min
    (a wrong p_min, or a node shifted by one spacing, planted in the oracle fails it)."""
    rho_s, p_s, _ = _isentrope_until(eos, w, lambda r, e, f: f + u)
    wl, wr = (w[0], -u, w[2]), (w[0], u, w[2])
    (ps, us, rl, rr), _ = O.riemann(eos, wl, eos, wr)
    K0 = eos.prm[0] * eos.prm[1] ** 2
    assert ps == pytest.approx(p_s, rel=1e-9, abs=1e-10 * K0)
    assert abs(us) <= 1e-9 * u
    assert rl == pytest.approx(rho_s, rel=1e-9) and rr == pytest.approx(rho_s, rel=1e-9)
    if eos is MGW_CUT:
        assert K0 * eos.prm[5] < ps < 0.0


@pytest.mark.parametrize("w,p", [((1000.0, 0.0, 1e5), 1e8), ((1000.0, 0.0, 1e5), 2e9), ((1100.0, 50.0, 3e8), 5e9),
                                 ((1000.0, 0.0, 1e5), 3e11)])
def test_mg_shock_curve_slope_is_the_derivative_of_the_curve(w, p):
    """The slope the MG shock branch returns (it drives the Newton iteration of the exact
    solver, Sec. 4.2) equals a central difference of the returned velocity change; d rho/dp on
    the Hugoniot comes from implicit differentiation of the energy equation, whose de/drho|_p a
    sign error planted in the oracle spoils."""
    f, df, _ = O.wave_curve(MGW, w, p)
    dp = 1e-5 * (p - w[2])
    fp, _, _ = O.wave_curve(MGW, w, p + dp)
    fm, _, _ = O.wave_curve(MGW, w, p - dp)
    assert df == pytest.approx((fp - fm) / (2 * dp), rel=1e-6)


@pytest.mark.parametrize("w", [(1000.0, 0.0, 1e5), (1243.0, 30.0, 1e9)])
def test_mg_wave_curve_slope_at_the_side_pressure(w):
    """At p = p_K the two branches of the MG wave curve meet with the acoustic slope 1/(rho c),
    which the curve returns there: a central difference across p_K (shock above, rarefaction
    below) gives the same slope."""
    f, df, rho = O.wave_curve(MGW, w, w[2])
    assert f == 0.0 and rho == w[0]
    dp = 1e-6 * w[2]
    fp, _, _ = O.wave_curve(MGW, w, w[2] + dp)
    fm, _, _ = O.wave_curve(MGW, w, w[2] - dp)
    assert df == pytest.approx((fp - fm) / (2 * dp), rel=1e-6)
    assert df == pytest.approx(1.0 / (w[0] * math.sqrt(O.sound_speed2(MGW, w[0], w[2]))), rel=1e-14)


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


def _boundary(pred, lo, hi, iters=200):
    """Bisection for the point where pred changes between lo (pred true) and hi (pred false)."""
    assert pred(lo) and not pred(hi)
    for _ in range(iters):
        mid = 0.5 * (lo + hi)
        if pred(mid):
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


@pytest.mark.parametrize("eL,wL,eR,wR,shocks", [
    (WATER, (1000.0, 0.0, 1e9), AIR, (1.0, 0.0, 1e5), (False, True)),     # stiffened fan | shock
    (AIR, (1.0, 0.0, 1e5), WATER, (1000.0, 0.0, 1e9), (True, False)),     # shock | stiffened fan
    (AIR, (1.0, 200.0, 1e5), AIR, (1.0, -200.0, 1e5), (True, True)),      # two shocks
    (AIR, (1.0, -100.0, 1e5), WATER, (1000.0, 100.0, 1e7), (False, False)),  # two fans
])
def test_exact_sampler_waves_satisfy_their_relations(eL, wL, eR, wR, shocks):
    """The exact two-stiffened-gas solution that the shock-tube convergence test measures
    against: each shock, located by bisection on xi = x/t, moves at the speed that carries the
    mass, momentum and energy jumps between the outer and the star state; each fan starts at
    u_K -+ c_K and ends at u* -+ c*_K, and inside it the state keeps (p + p_c)/rho^gamma and the
    Riemann invariant u +- 2c/(gamma - 1) of its side and sits on the characteristic xi = u -+ c."""
    def sample(xi):
        out, _ = O.exact_sample_sg(eL.prm, wL, eR.prm, wR, np.array([xi]))
        return out[:, 0]
    _, (ps, us, rls, rrs) = O.exact_sample_sg(eL.prm, wL, eR.prm, wR, np.zeros(1))
    for eos, w, rs, sgn, shock in ((eL, wL, rls, -1.0, shocks[0]), (eR, wR, rrs, 1.0, shocks[1])):
        g, pc = eos.prm
        assert (ps > w[2]) == shock
        c = math.sqrt(g * (w[2] + pc) / w[0])
        far = us + sgn * 10.0 * (abs(w[1]) + c + abs(us))

        def outer(xi):
            return np.array_equal(sample(xi), np.array(w))

        def star(xi):
            q = sample(xi)
            return q[0] == rs and q[1] == us and q[2] == ps
        if shock:
            S = _boundary(outer, far, us + sgn * 1e-9)
            assert star(S - sgn * 1e-9 * abs(S)) and outer(S + sgn * 1e-9 * abs(S))
            for res in _rh_residuals(lambda r, p: _e_sg(eos, r, p), w, (rs, us, ps)):
                assert res < 1e-12
            S_rh = (rs * us - w[0] * w[1]) / (rs - w[0])   # the speed the jumps require
            assert S == pytest.approx(S_rh, rel=1e-9)
        else:
            head = _boundary(outer, far, us + sgn * 1e-9)
            tail = _boundary(star, us + sgn * 1e-9, head)
            cs = math.sqrt(g * (ps + pc) / rs)
            assert head == pytest.approx(w[1] + sgn * c, rel=1e-9, abs=1e-9 * c)
            assert tail == pytest.approx(us + sgn * cs, rel=1e-9, abs=1e-9 * c)
            ent = (w[2] + pc) / w[0] ** g
            inv = w[1] - sgn * 2.0 * c / (g - 1.0)
            for f in (0.1, 0.37, 0.5, 0.81, 0.95):
                xi = tail + f * (head - tail)
                rho, u, p = sample(xi)
                cf = math.sqrt(g * (p + pc) / rho)
                assert (p + pc) / rho ** g == pytest.approx(ent, rel=1e-11)
                assert u - sgn * 2.0 * cf / (g - 1.0) == pytest.approx(inv, rel=1e-11, abs=1e-9 * c)
                assert u + sgn * cf == pytest.approx(xi, rel=1e-11, abs=1e-9 * c)


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


@pytest.mark.parametrize("vel", [(37.0, -23.0, 11.0), (-19.0, 29.0, -13.0)])
def test_level_set_residual_of_a_quartic_in_every_axis(vel):
    """L = -((u phi_x + v phi_y) + w phi_z) (Eq. levelset) with the third-order upwind-biased
    derivative of Sec. 4.4 along each axis: on phi = quartic(x) + quartic(y) + quartic(z) in a
    uniform flow each derivative is exact up to its truncation term, which for the stencil of a
    positive velocity is +(h^3/12) phi and for the other -(h^3/12) phi (Taylor
    expansion), so the residual checks the sign of every velocity term and that each axis is
    upwinded by its own velocity component."""
    n = (12, 12, 12)
    h = 1.0 / 12
    s = WL.Setup("quartic", n, h, (WL.WATER_SG, WL.AIR_PG), (0,) * 6, np.ones((12, 12, 12)),
                 np.zeros((12, 12, 12), np.uint8), {})
    x, y, z = WL.cell_centres(n, h)
    coef = {"x": (0.3, -0.4, 0.7, 0.2), "y": (-0.2, 0.5, -0.3, 0.1), "z": (0.25, 0.1, 0.4, -0.3)}

    def q(t, c):          # c4 t^4 + c3 t^3 + c2 t^2 + c1 t, t about 0.4
        t = t - 0.4
        return ((c[0] * t + c[1]) * t + c[2]) * t * t + c[3] * t

    def dq(t, c):
        t = t - 0.4
        return ((4 * c[0] * t + 3 * c[1]) * t + 2 * c[2]) * t + c[3]
    phi = 2.0 + q(x, coef["x"]) + q(y, coef["y"]) + q(z, coef["z"])
    P = np.zeros((5,) + phi.shape)
    P[0], P[1], P[2], P[3], P[4] = 1000.0, vel[0], vel[1], vel[2], 1e8
    g = _grid(s)
    _, L, _ = O.residual(g, O.prims_to_cons(g, P, phi), phi)
    D = [dq(t, coef[a]) + math.copysign(1.0, v) * h ** 3 / 12.0 * 24.0 * coef[a][0]
         for t, a, v in ((x, "x", vel[0]), (y, "y", vel[1]), (z, "z", vel[2]))]
    expect = -((vel[0] * D[0] + vel[1] * D[1]) + vel[2] * D[2])
    inner = (slice(2, -2),) * 3
    assert np.abs(L[inner] - expect[inner]).max() < 1e-9
    # the truncation terms are well above that bound: the wrong upwind choice on any axis fails
    assert min(abs(v) for v in vel) * 2 * h ** 3 / 12.0 * 24.0 * 0.2 > 1e-3


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


def test_two_reinit_iterations_in_closed_form():
    """Two iterations of Eq. reinit on phi0 = 2 (x - 0.43) evaluated by hand: the first moves
    each cell by (h/2) s_i with s_i = S(phi0_i) = phi0_i/sqrt(phi0_i^2 + h^2); the second takes
    the upwind one-sided slope of that iterate (the left one where phi0 >= 0, the right one
    where phi0 < 0; both positive here) as |grad phi|, and the same s_i: the smoothed sign
    stays that of phi0, not of the iterate."""
    n, h = (20, 4, 4), 1.0 / 20
    g = O.Grid(n=n, h=h, eos=(O.EOS(*WL.WATER_SG), O.EOS(*WL.AIR_PG)), bc=(0,) * 6)
    x, _, _ = WL.cell_centres(n, h)
    phi0 = 2.0 * (x[0, 0] - 0.43)
    s = phi0 / np.sqrt(phi0 * phi0 + h * h)
    frozen = np.zeros(20, bool)
    frozen[[8, 9]] = True
    phi1 = np.where(frozen, phi0, phi0 - 0.5 * h * s)
    left = np.empty(20)
    left[1:] = (phi1[1:] - phi1[:-1]) / h
    right = np.empty(20)
    right[:-1] = (phi1[1:] - phi1[:-1]) / h
    G = np.where(phi0 >= 0.0, left, right)
    cells = np.arange(1, 19)
    cells = cells[~frozen[cells]]
    expect = phi1[cells] - 0.5 * h * s[cells] * (G[cells] - 1.0)
    out = O.reinit(g, 2.0 * (x - 0.43), 2)
    assert np.abs(out[..., cells] - expect).max() < 1e-14
    assert np.array_equal(out[..., frozen], (2.0 * (x - 0.43))[..., frozen])


def test_reinit_keeps_a_distance_with_ridges():
    """The signed distance to two parallel planes on a periodic domain has a ridge (a kink of
    |grad phi| = 1 with the two one-sided slopes of opposite sign) in the middle of each phase,
    here on cell centres. It is a fixed point of the reinitialisation (Eq. reinit): the
    Godunov upwind norm of Sec. 4.4 takes the larger of the two admissible one-sided slopes
    along an axis, not their sum, so at a ridge it is still 1 (a sum planted in the oracle
    moves both ridges)."""
    n, h = (32, 4, 4), 1.0 / 32
    g = O.Grid(n=n, h=h, eos=(O.EOS(*WL.WATER_SG), O.EOS(*WL.AIR_PG)), bc=(1, 1, 0, 0, 0, 0))
    x, _, _ = WL.cell_centres(n, h)
    a, b = 9.2 * h, 23.8 * h      # ridges at x = 16.5 h (inside) and 0.5 h (outside, periodic)

    def dper(t):
        d = np.abs(x - t)
        return np.minimum(d, 1.0 - d)
    phi = np.where((x > a) & (x < b), -np.minimum(x - a, b - x), np.minimum(dper(a), dper(b)))
    out = O.reinit(g, phi, 5)
    assert np.abs(out - phi).max() < 1e-13


def test_one_reinit_iteration_in_closed_form():
    """One pseudo-time iteration of Eq. reinit on phi = 2 (x - 0.43) (|grad phi| = 2): away from
    the frozen first layer every cell moves by dtau S(phi0) (G - 1) with G = 2 (the upwind
    one-sided slopes), dtau = h/2 and S = phi0 / sqrt(phi0^2 + h^2) (Reading R24), all values
    read from the previous iterate (Jacobi)."""
    n, h = (20, 4, 4), 1.0 / 20
    g = O.Grid(n=n, h=h, eos=(O.EOS(*WL.WATER_SG), O.EOS(*WL.AIR_PG)), bc=(0,) * 6)
    x, _, _ = WL.cell_centres(n, h)
    phi = 2.0 * (x - 0.43)
    out = O.reinit(g, phi, 1)
    expect = phi - 0.5 * h * phi / np.sqrt(phi * phi + h * h) * (2.0 - 1.0)
    moving = np.ones(n[0], bool)
    moving[[8, 9]] = False        # the first layer: cells 8 (phi < 0) and 9 (phi > 0)
    assert np.abs(out[..., moving] - expect[..., moving]).max() < 1e-14
    assert np.array_equal(out[..., ~moving], phi[..., ~moving])


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
