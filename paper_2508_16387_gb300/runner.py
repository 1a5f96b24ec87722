"""Helpers that turn a workload Setup into a solver context on the GPU."""
from __future__ import annotations

from . import m2c as M


def grid_for(setup, precision=M.FP64, stream=None, device="cuda"):
    """A context for `setup` with its initial state built on the device: the post-shock
    Rankine-Hugoniot state from the library's Riemann solver, then primitives -> conserved."""
    g = M.Grid(setup.n, setup.h, setup.bc, setup.eos, precision=precision, cfl=setup.cfl,
               reinit_every=setup.reinit_every, reinit_iters=setup.reinit_iters, device=device, stream=stream)
    shocked = None
    if setup.shock is not None:
        amb = setup.prims_by_region[setup.shock[1]]
        r1, u1, _ = M.m2c_shock_state(setup.eos[0], (amb[0], amb[1], amb[4]), setup.shock[0])
        shocked = (r1, u1)
    g.set_prims(setup.prims(shocked), setup.phi)
    return g
