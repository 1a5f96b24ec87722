"""Seeded synthetic inputs for the solver and for the oracle.

This module holds no arithmetic of the method: it lays out grids, level sets
(signed distances) and piecewise-constant primitive states, and draws the
random parameters of the batched and served workloads. The one state that
needs the equation of state, the post-shock Rankine-Hugoniot state, is left as
a hole (region ``SHOCKED``) that each consumer fills with its own solver.

Workloads (the shock-bubble family restates the shock-induced bubble collapse
problem of the paper's Sec. 5.5 on a Cartesian box):

* ``shock_tube``: 1D two-material shock tube on nx x 4 x 4 cells, water
  (stiffened gas) at 1e9 Pa for x < 0.5 and air at 1e5 Pa for x > 0.5,
  phi = x - 0.5, transmissive in x and periodic in y and z.
* ``shock_bubble``: unit cube of water at 1e5 Pa with an air bubble
  (phi = |x - c| - R, air inside) and a planar shock at x = 0.2 whose post-shock
  pressure is given; transmissive on all sides.
* ``batched_instances``: many shock-bubble instances with random edge, radius,
  centre and shock pressure.
* ``served_trace``: a Poisson arrival trace of shock-bubble jobs.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Optional

import numpy as np

EOS_SG = 0
EOS_MG = 1
BC_TRANSMISSIVE = 0
BC_PERIODIC = 1

# region labels of the piecewise-constant initial state
AMBIENT = 0
BUBBLE = 1
SHOCKED = 2

# material parameters of the workloads (SI units)
WATER_SG = (EOS_SG, (6.12, 3.43e8))                         # stiffened gas
WATER_MG = (EOS_MG, (1000.0, 1483.0, 1.75, 0.28, 0.0, -math.inf))  # Mie-Grueneisen
AIR_PG = (EOS_SG, (1.4, 0.0))                                # perfect gas
EOS_NASG, EOS_JWL = 2, 3
# synthetic Noble-Abel stiffened-gas liquid (gamma, p_c, b, e_c) and detonation products
# (JWL: omega, A1, A2, R1, R2, rho0); parameter sets of the size such materials have
LIQUID_NASG = (EOS_NASG, (1.5, 5.0e8, 5.0e-4, -1.0e6))
PRODUCTS_JWL = (EOS_JWL, (0.3, 4.0e11, 4.0e9, 4.5, 1.0, 1600.0))


@dataclass
class Setup:
    """A grid, its two materials and a piecewise-constant initial state.

    ``eos[0]`` is the material where phi >= 0, ``eos[1]`` where phi < 0.
    ``prims_by_region[r]`` is (rho, u, v, w, p) for region r, except that the
    SHOCKED region is described by ``shock`` = (post-shock pressure, region of
    the state ahead of the shock) and is filled by the consumer.
    """
    name: str
    n: tuple                      # (nx, ny, nz)
    h: float
    eos: tuple                    # ((type, prm), (type, prm))
    bc: tuple                     # (x-, x+, y-, y+, z-, z+)
    phi: np.ndarray               # (nz, ny, nx) float64
    region: np.ndarray            # (nz, ny, nx) uint8
    prims_by_region: dict
    shock: Optional[tuple] = None
    cfl: float = 0.5
    reinit_every: int = 10
    reinit_iters: int = 5
    steps: int = 100
    meta: dict = field(default_factory=dict)

    @property
    def shape(self):
        return (self.n[2], self.n[1], self.n[0])

    @property
    def ncells(self) -> int:
        return self.n[0] * self.n[1] * self.n[2]

    def prims(self, shocked_state=None) -> np.ndarray:
        """Primitive fields (5, nz, ny, nx); ``shocked_state`` = (rho1, u1) of the
        post-shock state, computed by the consumer's own EOS code."""
        P = np.zeros((5,) + self.shape)
        for r, q in self.prims_by_region.items():
            m = self.region == r
            for v in range(5):
                P[v][m] = q[v]
        if self.shock is not None:
            m = self.region == SHOCKED
            if m.any():
                if shocked_state is None:
                    raise ValueError("the shocked region needs the post-shock state")
                rho1, u1 = shocked_state
                p1 = self.shock[0]
                P[0][m] = rho1
                P[1][m] = u1
                P[2][m] = 0.0
                P[3][m] = 0.0
                P[4][m] = p1
        return P


def cell_centres(n: tuple, h: float, lo=(0.0, 0.0, 0.0)):
    """Cell-centre coordinates (x, y, z), each of shape (nz, ny, nx): x_i = lo + (i + 1/2) h."""
    xs = lo[0] + (np.arange(n[0]) + 0.5) * h
    ys = lo[1] + (np.arange(n[1]) + 0.5) * h
    zs = lo[2] + (np.arange(n[2]) + 0.5) * h
    z, y, x = np.meshgrid(zs, ys, xs, indexing="ij")
    return x, y, z


def shock_tube(nx: int = 128, ny: int = 4, nz: int = 4, steps: int = 200) -> Setup:
    """Water (stiffened gas, 1e9 Pa) | air (perfect gas, 1e5 Pa) at x = 0.5, dx = 1/nx."""
    h = 1.0 / nx
    x, _, _ = cell_centres((nx, ny, nz), h)
    phi = x - 0.5
    region = np.where(phi < 0.0, BUBBLE, AMBIENT).astype(np.uint8)  # BUBBLE = water here (phi < 0)
    return Setup(
        name=f"shock_tube_{nx}x{ny}x{nz}",
        n=(nx, ny, nz), h=h,
        eos=(AIR_PG, WATER_SG),
        bc=(BC_TRANSMISSIVE, BC_TRANSMISSIVE, BC_PERIODIC, BC_PERIODIC, BC_PERIODIC, BC_PERIODIC),
        phi=phi, region=region,
        prims_by_region={AMBIENT: (1.0, 0.0, 0.0, 0.0, 1e5), BUBBLE: (1000.0, 0.0, 0.0, 0.0, 1e9)},
        steps=steps,
        meta={"left": (1000.0, 0.0, 1e9), "right": (1.0, 0.0, 1e5)},
    )


def shock_bubble(n: int = 128, radius: float = 0.15, centre=(0.5, 0.5, 0.5), p_shock: float = 1e9,
                 x_shock: float = 0.2, water=WATER_SG, steps: int = 500, name: Optional[str] = None) -> Setup:
    """Unit cube of water (1000 kg/m^3, 1e5 Pa) with an air bubble (1.2 kg/m^3, 1e5 Pa) and a
    planar shock at x_shock moving +x whose post-shock pressure is p_shock. Bubble cells take
    precedence over the shocked region."""
    h = 1.0 / n
    x, y, z = cell_centres((n, n, n), h)
    phi = np.sqrt((x - centre[0]) ** 2 + (y - centre[1]) ** 2 + (z - centre[2]) ** 2) - radius
    region = np.full(phi.shape, AMBIENT, dtype=np.uint8)
    region[x < x_shock] = SHOCKED
    region[phi < 0.0] = BUBBLE
    return Setup(
        name=name or f"shock_bubble_{n}^3",
        n=(n, n, n), h=h,
        eos=(water, AIR_PG),
        bc=(BC_TRANSMISSIVE,) * 6,
        phi=phi, region=region,
        prims_by_region={AMBIENT: (1000.0, 0.0, 0.0, 0.0, 1e5), BUBBLE: (1.2, 0.0, 0.0, 0.0, 1e5)},
        shock=(p_shock, AMBIENT),
        steps=steps,
        meta={"radius": radius, "centre": tuple(centre), "p_shock": p_shock, "x_shock": x_shock},
    )


@dataclass
class InstanceParams:
    edge: int
    radius: float
    centre: tuple
    p_shock: float
    steps: int = 200


def draw_instances(count: int = 64, seed: int = 3, edges=(32, 48, 64, 96, 128), steps: int = 200):
    """Parameters of ``count`` shock-bubble instances: edge uniform over ``edges``, radius
    U(0.08, 0.2), centre 0.5 + U(-0.1, 0.1) per axis, shock pressure log-uniform on [1e8, 2e9]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for _ in range(count):
        edge = int(rng.choice(np.asarray(edges)))
        radius = float(rng.uniform(0.08, 0.2))
        centre = tuple(float(0.5 + rng.uniform(-0.1, 0.1)) for _ in range(3))
        p_shock = float(math.exp(rng.uniform(math.log(1e8), math.log(2e9))))
        out.append(InstanceParams(edge, radius, centre, p_shock, steps))
    return out


def batched_instances(count: int = 64, seed: int = 3, water=WATER_SG, edges=(32, 48, 64, 96, 128),
                      steps: int = 200):
    """Setups of the batched workload (uneven cubic grids)."""
    return [shock_bubble(q.edge, q.radius, q.centre, q.p_shock, water=water, steps=q.steps,
                         name=f"instance{i}_{q.edge}^3")
            for i, q in enumerate(draw_instances(count, seed, edges, steps))]


@dataclass
class Job:
    job_id: int
    arrival: float          # seconds after the trace start
    params: InstanceParams


def served_trace(n_jobs: int = 200, rate: float = 20.0, seed: int = 4, edge_range=(48, 192),
                 steps_range=(100, 1000)):
    """Poisson arrivals at ``rate`` jobs/s; edge log-uniform on ``edge_range`` (rounded), steps
    uniform on the integers of ``steps_range``, the other parameters as in the batched workload."""
    rng = np.random.Generator(np.random.PCG64(seed))
    t = 0.0
    jobs = []
    for j in range(n_jobs):
        t += float(rng.exponential(1.0 / rate))
        edge = int(round(math.exp(rng.uniform(math.log(edge_range[0]), math.log(edge_range[1])))))
        steps = int(rng.integers(steps_range[0], steps_range[1] + 1))
        radius = float(rng.uniform(0.08, 0.2))
        centre = tuple(float(0.5 + rng.uniform(-0.1, 0.1)) for _ in range(3))
        p_shock = float(math.exp(rng.uniform(math.log(1e8), math.log(2e9))))
        jobs.append(Job(j, t, InstanceParams(edge, radius, centre, p_shock, steps)))
    return jobs


def random_state(n: tuple, seed: int, eos=(WATER_SG, AIR_PG), two_phase: bool = True, amp: float = 0.05,
                 base=None):
    """Smooth random single- or two-material test state on an (nx, ny, nz) grid with h = 1/nx:
    primitive fields of moderate amplitude around reference states (density, pressure) of
    material 0 (phi >= 0) and 1 (phi < 0), water- and air-like unless ``base`` = {0: (rho, p),
    1: (rho, p)} gives others, and a level set that is a randomly placed sphere (two_phase) or
    all positive."""
    rng = np.random.Generator(np.random.PCG64(seed))
    h = 1.0 / n[0]
    x, y, z = cell_centres(n, h)
    shape = x.shape
    if two_phase:
        c = rng.uniform(0.3, 0.7, size=3) * np.array([n[0], n[1], n[2]]) * h
        r = 0.25 * min(n) * h
        phi = np.sqrt((x - c[0]) ** 2 + (y - c[1]) ** 2 + (z - c[2]) ** 2) - r
    else:
        phi = np.ones(shape)
    P = np.zeros((5,) + shape)
    base = base or {0: (1000.0, 1e8), 1: (1.2, 1e5)}
    vel = {0: 50.0, 1: 50.0}
    for m in (0, 1):
        sel = (phi < 0.0) if m == 1 else (phi >= 0.0)
        rho0, p0 = base[m]
        noise = rng.uniform(-1.0, 1.0, size=(5,) + shape)
        P[0][sel] = (rho0 * (1.0 + amp * noise[0]))[sel]
        for v in (1, 2, 3):
            P[v][sel] = (vel[m] * noise[v])[sel]
        P[4][sel] = (p0 * (1.0 + amp * noise[4]))[sel]
    return P, phi


def shock_bubble_device(n: int, radius: float, centre, p_shock: float, x_shock: float = 0.2, device="cuda"):
    """The fields of shock_bubble() built directly in device memory (torch, float64), for
    servers that create many grids: (phi, region) tensors of shape (n, n, n). The same
    formulas as shock_bubble(), so the fields are identical."""
    import torch
    h = 1.0 / n
    c = (torch.arange(n, dtype=torch.float64, device=device) + 0.5) * h
    z, y, x = torch.meshgrid(c, c, c, indexing="ij")
    phi = torch.sqrt((x - centre[0]) ** 2 + (y - centre[1]) ** 2 + (z - centre[2]) ** 2) - radius
    region = torch.full(phi.shape, AMBIENT, dtype=torch.uint8, device=device)
    region[x < x_shock] = SHOCKED
    region[phi < 0.0] = BUBBLE
    return phi, region


def prims_device(region, prims_by_region: dict, shocked_state=None, p_shock: float = 0.0):
    """Primitive fields (5, nz, ny, nx) on the device from a region map (see Setup.prims)."""
    import torch
    P = torch.zeros((5,) + tuple(region.shape), dtype=torch.float64, device=region.device)
    for r, q in prims_by_region.items():
        m = region == r
        for v in range(5):
            P[v][m] = q[v]
    if shocked_state is not None:
        m = region == SHOCKED
        P[0][m] = shocked_state[0]
        P[1][m] = shocked_state[1]
        P[2][m] = 0.0
        P[3][m] = 0.0
        P[4][m] = p_shock
    return P
