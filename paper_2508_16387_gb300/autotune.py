"""Autotuner of the bulk stage kernel's launch: tile shape (32 x 4, 32 x 8 or,
on the mixed path, 32 x 16 columns; z-length of a tile), tile schedule (fixed
stride or atomic counter) and persistent grid size, picked by timing candidates with CUDA events on the
actual grids. The state is saved before and restored after every trial, so
tuning leaves the simulation where it was, except that the exact Riemann
solver's warm-start star pressures start empty again (a restored state is a
new state), which moves later results by no more than the Newton tolerance.
The choice itself never changes a result (every cell is computed by the same
arithmetic under every tiling).
"""
from __future__ import annotations

import itertools
from dataclasses import dataclass

from . import m2c as M

DEFAULT_CANDIDATES = [(ty, tz, sched, bpsm) for ty, tz, sched, bpsm in
                      itertools.product((8, 16), (0, 16, 32), (0, 1), (0, 2, 4))
                      if not (sched == 1 and bpsm == 0)]
FP64_CANDIDATES = [(8, 0, 0, 0), (8, 0, 1, 1), (4, 0, 1, 2), (8, 32, 1, 1)]


@dataclass
class Trial:
    tuning: tuple
    ms_per_step: float


class _Saved:
    def __init__(self, grids):
        self.items = []
        for g in grids:
            t, step = g.sync()
            self.items.append((g, g.W.clone(), g.phi.clone(), t, step))

    def restore(self):
        for g, W, phi, t, step in self.items:
            g.W.copy_(W)
            g.phi.copy_(phi)
            g.set_state(None, None, t=t, step=step)


def _time(torch, fn, steps):
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    fn(steps)
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def tune_batch(grids, candidates=None, trial_steps=2, warm_steps=1):
    """Best (tile rows, tile z, schedule, blocks per SM) for stepping `grids` as one batch."""
    import torch
    saved = _Saved(grids)
    trials = []
    for tun in candidates or DEFAULT_CANDIDATES:
        b = M.Batch(grids, tun)
        b.step(warm_steps)
        ms = _time(torch, b.step, trial_steps)
        del b
        saved.restore()
        trials.append(Trial(tun, ms))
    trials.sort(key=lambda t: t.ms_per_step)
    return trials[0].tuning, trials


def tune_grid(grid, candidates=((8, 0), (4, 0), (8, 16), (8, 32), (4, 16), (4, 32)), trial_steps=2, warm_steps=1):
    """Best (tile rows, tile z) for stepping one grid with m2c_step."""
    import torch
    saved = _Saved([grid])
    trials = []
    for ty, tz in candidates:
        grid.set_tiling(ty, tz)
        grid.step(warm_steps)
        ms = _time(torch, grid.step, trial_steps)
        saved.restore()
        trials.append(Trial((ty, tz), ms))
    trials.sort(key=lambda t: t.ms_per_step)
    grid.set_tiling(*trials[0].tuning)
    return trials[0].tuning, trials
