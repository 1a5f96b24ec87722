"""Host logic of the autotuner with the device parts replaced by fakes (no GPU): every candidate
is tried, the fastest is returned with the trials sorted by time, and every trial starts from
(and the tuner leaves) the state, time and step count it found."""
import pytest

torch = pytest.importorskip("torch")

from paper_2508_16387_gb300 import autotune as AT  # noqa: E402


class FakeGrid:
    def __init__(self, k):
        self.W = torch.full((5, 2, 2, 2), float(k))
        self.phi = torch.full((2, 2, 2), -float(k))
        self.t, self.step = 0.25 * k, 10 + k

    def sync(self):
        return self.t, self.step

    def set_state(self, W, phi, t=0.0, step=0):
        self.t, self.step = t, step


def test_tune_batch_picks_the_fastest_and_restores_the_state(monkeypatch):
    cost = {(8, 0, 0, 0): 3.0, (16, 32, 1, 2): 1.5, (4, 16, 0, 4): 2.0}
    seen = []

    class FakeBatch:
        def __init__(self, grids, tuning):
            self.grids, self.tuning = grids, tuning
            seen.append((tuning, [(g.W.clone(), g.phi.clone(), g.t, g.step) for g in grids]))

        def step(self, n):          # changes every grid, as stepping does
            for g in self.grids:
                g.W += n
                g.phi -= n
                g.t += 0.1 * n
                g.step += n

    monkeypatch.setattr(AT.M, "Batch", FakeBatch)
    monkeypatch.setattr(AT, "_time", lambda torch_, fn, steps: (fn(steps), cost[fn.__self__.tuning])[1])
    grids = [FakeGrid(1), FakeGrid(2)]
    start = [(g.W.clone(), g.phi.clone(), g.t, g.step) for g in grids]
    best, trials = AT.tune_batch(grids, candidates=list(cost), trial_steps=3)
    assert best == (16, 32, 1, 2)
    assert [t.tuning for t in trials] == [(16, 32, 1, 2), (4, 16, 0, 4), (8, 0, 0, 0)]
    assert [t.ms_per_step for t in trials] == [1.5, 2.0, 3.0]
    assert [s[0] for s in seen] == list(cost)
    for _, states in seen:          # every trial started from the state the tuner found
        for (W, phi, t, step), (W0, phi0, t0, step0) in zip(states, start):
            assert torch.equal(W, W0) and torch.equal(phi, phi0) and (t, step) == (t0, step0)
    for g, (W0, phi0, t0, step0) in zip(grids, start):   # and it left that state behind
        assert torch.equal(g.W, W0) and torch.equal(g.phi, phi0) and (g.t, g.step) == (t0, step0)


def test_default_candidates_are_valid_launches():
    """Tile rows 4, 8 or 16; an atomic schedule only with a persistent grid; FP64 without 16 rows."""
    for ty, tz, sched, bpsm in AT.DEFAULT_CANDIDATES:
        assert ty in (4, 8, 16) and tz >= 0 and sched in (0, 1) and bpsm >= 0
        assert not (sched == 1 and bpsm == 0)
    assert all(c[0] in (4, 8) for c in AT.FP64_CANDIDATES)
