"""Error metrics of the parity tests (test helpers only).

conserved_errors reads "max relative error on conserved variables" normwise
(Reading R29): for the density and the total energy, max over cells of
|a - b| over max over cells of |b|; for the momentum, the same with the
Euclidean norm of the momentum vector (rho u, rho v, rho w), so that a
velocity component that is small everywhere (the transverse momentum of a
planar shock hitting a bubble) is measured on the scale of the momentum it
exchanges with, not on its own.
"""
import numpy as np


def conserved_errors(a, b):
    """[rho, momentum vector, rho E] errors of conserved states a, b of shape (5, ...)."""
    out = []
    for sel in ((0,), (1, 2, 3), (4,)):
        d = np.sqrt(sum((a[v] - b[v]) ** 2 for v in sel))
        n = np.sqrt(sum(b[v] ** 2 for v in sel))
        out.append(float(d.max() / max(n.max(), 1e-300)))
    return out
