"""Batched stepping (one launch per kernel for many uneven grids), CUDA-graph
capture and the autotuner: every grid's result is the same alone and in the
batch, bit for bit (each cell is computed by the same arithmetic)."""
import numpy as np
import pytest

from paper_2508_16387_gb300 import workloads as WL

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2508_16387_gb300 import m2c as M
    from paper_2508_16387_gb300 import runner as RN
    M.lib()
    return M, RN


def small_batch():
    params = WL.draw_instances(count=5, seed=7, edges=(16, 20, 24, 28, 32), steps=12)
    return [WL.shock_bubble(q.edge, q.radius, q.centre, q.p_shock, steps=q.steps) for q in params]


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("tuning", [(8, 0, 0, 0), (4, 8, 1, 2), (8, 16, 0, 1)])
def test_batch_equals_alone(env, prec, tuning):
    M, RN = env
    setups = small_batch()
    alone = []
    for s in setups:
        g = RN.grid_for(s, prec)
        g.step(12)
        g.sync()
        alone.append((g.W.cpu().numpy(), g.phi.cpu().numpy()))
    grids = [RN.grid_for(s, prec) for s in setups]
    b = M.Batch(grids, tuning)
    b.step(12)
    for g, (Wa, pa) in zip(grids, alone):
        t, k = g.sync()
        assert k == 12
        assert np.array_equal(g.W.cpu().numpy(), Wa)
        assert np.array_equal(g.phi.cpu().numpy(), pa)


def test_graph_replay_equals_eager(env):
    M, RN = env
    setups = small_batch()
    eager = [RN.grid_for(s, 1) for s in setups]
    be = M.Batch(eager, (8, 0, 1, 2))
    be.step(20)
    graphed = [RN.grid_for(s, 1) for s in setups]
    bg = M.Batch(graphed, (8, 0, 1, 2))
    bg.capture(10)
    bg.launch_graph()
    bg.launch_graph()
    for a, b in zip(eager, graphed):
        ta, ka = a.sync()
        tb, kb = b.sync()
        assert ka == kb == 20 and ta == tb
        assert np.array_equal(a.W.cpu().numpy(), b.W.cpu().numpy())
    bg.capture(3)
    for _ in range(4):   # steps 20-31, reinitialisation after step 29 read on the device
        bg.launch_graph()
    be.step(12)
    for a, b in zip(eager, graphed):
        assert a.sync() == b.sync()
        assert np.array_equal(a.phi.cpu().numpy(), b.phi.cpu().numpy())


def test_autotuner_restores_state(env):
    M, RN = env
    from paper_2508_16387_gb300 import autotune as AT
    setups = small_batch()
    grids = [RN.grid_for(s, 1) for s in setups]
    W0 = [g.W.cpu().numpy() for g in grids]
    best, trials = AT.tune_batch(grids, candidates=[(8, 0, 0, 0), (4, 0, 1, 2), (8, 16, 0, 2)], trial_steps=2)
    assert best in [t.tuning for t in trials] and len(trials) == 3
    for g, w in zip(grids, W0):
        t, k = g.sync()
        assert k == 0 and t == 0.0
        assert np.array_equal(g.W.cpu().numpy(), w)


def test_grids_at_different_steps_batch_like_alone(env):
    """A grid that joins a batch at another step keeps its own reinitialisation schedule."""
    M, RN = env
    setups = small_batch()[:3]
    alone = []
    for s in setups:
        g = RN.grid_for(s, 0)
        g.step(17)
        g.sync()
        alone.append(g.W.cpu().numpy())
    grids = [RN.grid_for(s, 0) for s in setups]
    grids[0].step(7)          # grid 0 runs ahead by 7 steps, then all step together
    grids[1].step(3)
    b = M.Batch(grids, (8, 0, 0, 0))
    b.step(10)
    grids[1].step(4)
    grids[2].step(7)
    for g, w in zip(grids, alone):
        assert g.sync()[1] == 17
        assert np.array_equal(g.W.cpu().numpy(), w)
