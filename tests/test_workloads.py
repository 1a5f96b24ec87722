"""The seeded synthetic inputs follow their stated recipe (CPU): determinism per seed, parameter
ranges, arrival statistics of the served trace, the batched workload's size, and the geometry
of the shock-bubble and shock-tube setups."""
import math

import numpy as np

from paper_2508_16387_gb300 import workloads as WL


def test_instances_are_seeded_and_in_range():
    a, b = WL.draw_instances(64, seed=3), WL.draw_instances(64, seed=3)
    assert a == b and WL.draw_instances(64, seed=4) != a
    for q in a:
        assert q.edge in (32, 48, 64, 96, 128)
        assert 0.08 <= q.radius < 0.2
        assert all(0.4 <= c < 0.6 for c in q.centre)
        assert 1e8 <= q.p_shock <= 2e9
    # 64 draws of edge^3 with mean (32^3 + 48^3 + 64^3 + 96^3 + 128^3)/5 = 677,478 cells
    cells = sum(q.edge ** 3 for q in a)
    assert abs(cells / (64 * 677478) - 1) < 0.25
    assert len({q.edge for q in a}) == 5


def test_served_trace_recipe():
    jobs = WL.served_trace(200, rate=20.0, seed=4)
    assert jobs == WL.served_trace(200, rate=20.0, seed=4)
    t = np.array([j.arrival for j in jobs])
    assert np.all(np.diff(t) > 0) and t[0] > 0
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert abs(gaps.mean() * 20.0 - 1) < 0.2                     # Poisson at 20 jobs/s
    assert abs(gaps.std() / gaps.mean() - 1) < 0.25              # exponential gaps
    edges = np.array([j.params.edge for j in jobs])
    steps = np.array([j.params.steps for j in jobs])
    assert edges.min() >= 48 and edges.max() <= 192 and steps.min() >= 100 and steps.max() <= 1000
    # log-uniform edges: the median edge is near sqrt(48 * 192) = 96
    assert abs(np.median(edges) / 96 - 1) < 0.2
    assert [j.job_id for j in jobs] == list(range(200))


def test_shock_bubble_geometry():
    s = WL.shock_bubble(n=32, radius=0.2, centre=(0.5, 0.45, 0.55), x_shock=0.3)
    x, y, z = WL.cell_centres(s.n, s.h)
    d = np.sqrt((x - 0.5) ** 2 + (y - 0.45) ** 2 + (z - 0.55) ** 2)
    assert np.allclose(s.phi, d - 0.2, rtol=0, atol=1e-15)       # signed distance to the sphere
    assert np.array_equal(s.region == WL.BUBBLE, s.phi < 0)      # bubble cells win
    assert np.array_equal(s.region == WL.SHOCKED, (x < 0.3) & (s.phi >= 0))
    assert s.bc == (WL.BC_TRANSMISSIVE,) * 6 and s.shock[1] == WL.AMBIENT
    assert s.prims_by_region[WL.BUBBLE][0] == 1.2 and s.prims_by_region[WL.AMBIENT][0] == 1000.0


def test_shock_tube_geometry():
    s = WL.shock_tube(nx=64, ny=4, nz=4)
    x, _, _ = WL.cell_centres(s.n, s.h)
    assert np.array_equal(s.phi, x - 0.5)
    assert s.eos[1] == WL.WATER_SG and s.eos[0] == WL.AIR_PG     # water where phi < 0
    assert s.bc[:2] == (WL.BC_TRANSMISSIVE,) * 2 and s.bc[2:] == (WL.BC_PERIODIC,) * 4
    assert math.isclose(s.h, 1 / 64)


def test_random_state_is_seeded():
    P1, phi1 = WL.random_state((12, 10, 8), seed=5)
    P2, phi2 = WL.random_state((12, 10, 8), seed=5)
    assert np.array_equal(P1, P2) and np.array_equal(phi1, phi2)
    assert (phi1 < 0).any() and (phi1 >= 0).any()
    assert np.all(P1[0] > 0) and np.all(P1[4] > 0)
