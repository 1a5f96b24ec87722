"""ctypes binding of the CPU FP64 oracle (``m2c_oracle.c``).

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers. Nothing in the GPU
solver package imports this module, and this module imports nothing from it.

All arrays are float64 numpy arrays in structure-of-arrays layout with x
fastest: a conserved state ``W`` has shape ``(5, nz, ny, nx)``, a level set
``phi`` has shape ``(nz, ny, nx)``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "m2c_oracle.c")
LIB = os.path.join(HERE, "libm2c_oracle.so")
# a prebuilt copy of the oracle to load instead (the mutation test builds copies with a planted
# mistake and runs pins against them); unset: the library built from SRC above
MUTANT_LIB = os.environ.get("M2C_ORACLE_MUTANT_LIB", "")
CFLAGS = ["-O2", "-std=c11", "-ffp-contract=off", "-fopenmp", "-shared", "-fPIC"]

EOS_SG = 0
EOS_MG = 1
EOS_NASG = 2  # Noble-Abel stiffened gas, prm = (gamma, p_c, b, e_c)
EOS_JWL = 3  # Jones-Wilkins-Lee, prm = (omega, A1, A2, R1, R2, rho0)
BC_TRANSMISSIVE = 0
BC_PERIODIC = 1
BC_SYMMETRY = 2  # mirror side: the normal velocity is negated in the ghost cells
GEOM_CARTESIAN, GEOM_CYLINDRICAL, GEOM_SPHERICAL = 0, 1, 2  # x is the radius in the last two
LIM_VA_MOD, LIM_MC = 0, 1
FLUX_HLLC, FLUX_LLF = 0, 1

STATUS = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 4: "ENOCONV", 5: "ENONPHYS", 6: "EVACUUM"}


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction, OpenMP over cells)."""
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        subprocess.run(["gcc", *CFLAGS, "-o", LIB, SRC, "-lm"], check=True)
    return LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        if MUTANT_LIB:
            _lib = ctypes.CDLL(MUTANT_LIB)
        else:
            build()
            _lib = ctypes.CDLL(LIB)
        d = ctypes.c_double
        p = ctypes.c_void_p
        i = ctypes.c_int
        L = ctypes.c_long
        _lib.or_va_slope.restype = d
        _lib.or_va_slope.argtypes = [d, d]
        _lib.or_mc_slope.restype = d
        _lib.or_mc_slope.argtypes = [d, d, d]
        _lib.or_band_cutoff.restype = d
        _lib.or_band_cutoff.argtypes = [d, d, d, d]
        _lib.or_llf.argtypes = [i, p, p, p, i, p]
        for name in ("or_eos_pressure", "or_eos_energy", "or_eos_c2"):
            getattr(_lib, name).argtypes = [i, p, d, d, p]
        _lib.or_wave_curve.argtypes = [i, p, p, d, p]
        _lib.or_riemann.argtypes = [i, p, p, i, p, p, p, p]
        _lib.or_riemann_batch.argtypes = [i, i, p, p, i, p, p, p, p, p]
        _lib.or_hllc.argtypes = [i, p, p, p, i, p]
        _lib.or_shock_state.argtypes = [i, p, p, d, p]
        _lib.or_prims_to_cons.argtypes = [p, p, p, p, p]
        _lib.or_cons_to_prims.argtypes = [p, p, p, p, p]
        _lib.or_time_step.argtypes = [p, p, p, p, p]
        _lib.or_residual.argtypes = [p, p, p, p, p, p, p]
        _lib.or_run.argtypes = [p, p, p, p, L, i, p, p, p]
        _lib.or_reinit.argtypes = [p, p, p, i]
        _lib.or_phase_fix.argtypes = [p, p, p, p, p, p]
        _lib.or_exact_sample_sg.argtypes = [p, p, p, p, i, p, p, p]
        _lib.or_num_threads.restype = i
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


class OracleError(RuntimeError):
    def __init__(self, code: int, where: str = ""):
        super().__init__(f"oracle {where}: {STATUS.get(code, code)}")
        self.code = code


def _check(code: int, where: str):
    if code != 0:
        raise OracleError(code, where)


def _f64(x, n=None) -> np.ndarray:
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float64))
    if n is not None:
        assert a.size == n
    return a


@dataclass
class EOS:
    """An equation of state: ``type`` EOS_SG with prm = (gamma, p_c) or EOS_MG with
    prm = (rho0, c0, s, Gamma0, e0, eta_min)."""
    type: int
    prm: tuple

    def arr(self) -> np.ndarray:
        a = np.zeros(6)
        a[: len(self.prm)] = self.prm
        if self.type == EOS_MG and len(self.prm) < 6:
            a[5] = -np.inf
        return a


@dataclass
class Grid:
    n: tuple  # (nx, ny, nz)
    h: float
    eos: tuple  # (eos for phi >= 0, eos for phi < 0)
    bc: tuple = (0, 0, 0, 0, 0, 0)
    cfl: float = 0.5
    reinit_every: int = 10
    reinit_iters: int = 5
    threads: int = 0  # 0: OpenMP default
    rk: int = 2  # Runge-Kutta order of Sec. 4.3: 2 (TVD RK2), 3 (TVD RK3), 1 (forward Euler)
    limiter: int = 0  # LIM_VA_MOD or LIM_MC (App. D)
    flux: int = 0  # FLUX_HLLC or FLUX_LLF (App. C)
    mc_alpha: float = 1.2  # alpha of the MC limiter
    dt_fixed: float = 0.0  # > 0: constant time step instead of the CFL rule (Sec. 4.3)
    geom: int = 0  # GEOM_CARTESIAN, GEOM_CYLINDRICAL (x = r, z axial; ny = 1) or GEOM_SPHERICAL (x = r; 1D)
    x0: float = 0.0  # lower x coordinate (the radius of the first cell's lower face)
    band_beta: float = 0.0  # narrow-band level set (Reading R38): inner tube radius in cells
    band_gamma: float = 0.0  # outer tube radius in cells; 0 = the full domain

    def packed(self):
        ip = np.array(list(self.n) + list(self.bc) + [self.reinit_every, self.reinit_iters,
                      self.eos[0].type, self.eos[1].type, self.threads, self.rk, self.limiter, self.flux,
                      self.geom],
                      dtype=np.int32)
        dp = np.concatenate([[self.h, self.cfl], self.eos[0].arr(), self.eos[1].arr(),
                             [self.mc_alpha, self.dt_fixed, self.x0, self.band_beta, self.band_gamma]]
                            ).astype(np.float64)
        return ip, dp

    @property
    def shape(self):
        return (self.n[2], self.n[1], self.n[0])


def va_slope(a: float, b: float) -> float:
    return lib().or_va_slope(a, b)


def mc_slope(a: float, b: float, alpha: float = 1.2) -> float:
    return lib().or_mc_slope(a, b, alpha)


def band_cutoff(beta: float, gamma: float, h: float, phi: float) -> float:
    """Narrow-band cutoff of the level-set velocity (Reading R38); beta, gamma in cells."""
    return lib().or_band_cutoff(beta, gamma, h, phi)


def _eos_call(name, eos: EOS, x: float, y: float) -> float:
    out = np.zeros(1)
    _check(getattr(lib(), name)(eos.type, _ptr(eos.arr()), x, y, _ptr(out)), name)
    return float(out[0])


def pressure(eos: EOS, rho: float, e: float) -> float:
    return _eos_call("or_eos_pressure", eos, rho, e)


def energy(eos: EOS, rho: float, p: float) -> float:
    return _eos_call("or_eos_energy", eos, rho, p)


def sound_speed2(eos: EOS, rho: float, p: float) -> float:
    return _eos_call("or_eos_c2", eos, rho, p)


def wave_curve(eos: EOS, w, p: float):
    """(f, df/dp, rho behind the wave) of the wave taking w = (rho, u, p) to pressure p."""
    out = np.zeros(3)
    _check(lib().or_wave_curve(eos.type, _ptr(eos.arr()), _ptr(_f64(w, 3)), p, _ptr(out)), "wave_curve")
    return tuple(out)


def riemann(eosL: EOS, wL, eosR: EOS, wR):
    """Exact two-material Riemann solution: ((p*, u*, rho*_L, rho*_R), iterations)."""
    out = np.zeros(4)
    it = np.zeros(1, dtype=np.int32)
    _check(lib().or_riemann(eosL.type, _ptr(eosL.arr()), _ptr(_f64(wL, 3)), eosR.type, _ptr(eosR.arr()),
                            _ptr(_f64(wR, 3)), _ptr(out), _ptr(it)), "riemann")
    return tuple(out), int(it[0])


def riemann_status(eosL: EOS, wL, eosR: EOS, wR) -> int:
    out = np.zeros(4)
    it = np.zeros(1, dtype=np.int32)
    return lib().or_riemann(eosL.type, _ptr(eosL.arr()), _ptr(_f64(wL, 3)), eosR.type, _ptr(eosR.arr()),
                            _ptr(_f64(wR, 3)), _ptr(out), _ptr(it))


def riemann_batch(eosL: EOS, L: np.ndarray, eosR: EOS, R: np.ndarray):
    """Batch of n problems, L and R of shape (3, n) = (rho, u, p). Returns (out (4, n), iters, status)."""
    L = _f64(L)
    R = _f64(R)
    n = L.shape[1]
    out = np.zeros((4, n))
    it = np.zeros(n, dtype=np.int32)
    stt = np.zeros(n, dtype=np.int32)
    lib().or_riemann_batch(n, eosL.type, _ptr(eosL.arr()), _ptr(L), eosR.type, _ptr(eosR.arr()), _ptr(R),
                           _ptr(out), _ptr(it), _ptr(stt))
    return out, it, stt


def hllc(eos: EOS, qL, qR, d: int) -> np.ndarray:
    F = np.zeros(5)
    _check(lib().or_hllc(eos.type, _ptr(eos.arr()), _ptr(_f64(qL, 5)), _ptr(_f64(qR, 5)), d, _ptr(F)), "hllc")
    return F


def llf(eos: EOS, qL, qR, d: int) -> np.ndarray:
    F = np.zeros(5)
    _check(lib().or_llf(eos.type, _ptr(eos.arr()), _ptr(_f64(qL, 5)), _ptr(_f64(qR, 5)), d, _ptr(F)), "llf")
    return F


def shock_state(eos: EOS, w, p1: float):
    """(rho1, u1, shock speed) behind a shock moving in +x into w = (rho, u, p) at pressure p1."""
    out = np.zeros(3)
    _check(lib().or_shock_state(eos.type, _ptr(eos.arr()), _ptr(_f64(w, 3)), p1, _ptr(out)), "shock_state")
    return tuple(out)


def prims_to_cons(g: Grid, prims: np.ndarray, phi: np.ndarray) -> np.ndarray:
    ip, dp = g.packed()
    prims = _f64(prims)
    phi = _f64(phi)
    W = np.zeros((5,) + g.shape)
    _check(lib().or_prims_to_cons(_ptr(ip), _ptr(dp), _ptr(prims), _ptr(phi), _ptr(W)), "prims_to_cons")
    return W


def cons_to_prims(g: Grid, W: np.ndarray, phi: np.ndarray) -> np.ndarray:
    ip, dp = g.packed()
    P = np.zeros((5,) + g.shape)
    _check(lib().or_cons_to_prims(_ptr(ip), _ptr(dp), _ptr(_f64(W)), _ptr(_f64(phi)), _ptr(P)), "cons_to_prims")
    return P


def time_step(g: Grid, W: np.ndarray, phi: np.ndarray) -> float:
    ip, dp = g.packed()
    dt = np.zeros(1)
    _check(lib().or_time_step(_ptr(ip), _ptr(dp), _ptr(_f64(W)), _ptr(_f64(phi)), _ptr(dt)), "time_step")
    return float(dt[0])


def residual(g: Grid, W: np.ndarray, phi: np.ndarray):
    """One stage residual: (R (5, nz, ny, nx), L (nz, ny, nx), stats)."""
    ip, dp = g.packed()
    R = np.zeros((5,) + g.shape)
    L = np.zeros(g.shape)
    st = np.zeros(3, dtype=np.int64)
    _check(lib().or_residual(_ptr(ip), _ptr(dp), _ptr(_f64(W)), _ptr(_f64(phi)), _ptr(R), _ptr(L), _ptr(st)),
           "residual")
    return R, L, {"interface_faces": int(st[0]), "newton_max": int(st[1])}


@dataclass
class RunResult:
    W: np.ndarray
    phi: np.ndarray
    t: float
    dts: np.ndarray
    stats: dict = field(default_factory=dict)


def run(g: Grid, W: np.ndarray, phi: np.ndarray, nsteps: int, step0: int = 0, t0: float = 0.0) -> RunResult:
    """Advance copies of (W, phi) by nsteps time steps."""
    ip, dp = g.packed()
    W = _f64(W).copy()
    phi = _f64(phi).copy()
    t = np.array([float(t0)])
    st = np.zeros(4, dtype=np.int64)
    dts = np.zeros(max(nsteps, 1))
    _check(lib().or_run(_ptr(ip), _ptr(dp), _ptr(W), _ptr(phi), step0, nsteps, _ptr(t), _ptr(st), _ptr(dts)), "run")
    return RunResult(W, phi, float(t[0]), dts[:nsteps],
                     {"interface_faces": int(st[0]), "newton_max": int(st[1]), "flipped": int(st[2])})


def run_status(g: Grid, W: np.ndarray, phi: np.ndarray, nsteps: int, step0: int = 0):
    """Like run() but returns (status code, err_cell) instead of raising."""
    ip, dp = g.packed()
    W = _f64(W).copy()
    phi = _f64(phi).copy()
    t = np.zeros(1)
    st = np.zeros(4, dtype=np.int64)
    code = lib().or_run(_ptr(ip), _ptr(dp), _ptr(W), _ptr(phi), step0, nsteps, _ptr(t), _ptr(st), None)
    return code, int(st[3])


def phase_fix(g: Grid, W: np.ndarray, phi: np.ndarray, id_old: np.ndarray):
    """The phase update alone on copies of (W, phi), given the material ids at the start of
    the step: returns (W, phi, number of cells that changed material)."""
    ip, dp = g.packed()
    W = _f64(W).copy()
    phi = _f64(phi).copy()
    ido = np.ascontiguousarray(id_old, dtype=np.uint8)
    nf = np.zeros(1, dtype=np.int64)
    _check(lib().or_phase_fix(_ptr(ip), _ptr(dp), _ptr(W), _ptr(phi), _ptr(ido), _ptr(nf)), "phase_fix")
    return W, phi, int(nf[0])


def reinit(g: Grid, phi: np.ndarray, iters: int) -> np.ndarray:
    ip, dp = g.packed()
    phi = _f64(phi).copy()
    _check(lib().or_reinit(_ptr(ip), _ptr(dp), _ptr(phi), iters), "reinit")
    return phi


def exact_sample_sg(prmL, wL, prmR, wR, xi: np.ndarray):
    """Exact solution of a two-stiffened-gas Riemann problem at xi = x/t: ((rho, u, p) arrays, star)."""
    xi = _f64(xi)
    n = xi.size
    out = np.zeros((3, n))
    star = np.zeros(4)
    _check(lib().or_exact_sample_sg(_ptr(_f64(prmL, 2)), _ptr(_f64(wL, 3)), _ptr(_f64(prmR, 2)), _ptr(_f64(wR, 3)),
                                    n, _ptr(xi), _ptr(out), _ptr(star)), "exact_sample_sg")
    return out, tuple(star)


def num_threads() -> int:
    return lib().or_num_threads()
