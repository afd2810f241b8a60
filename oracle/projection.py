"""Exact solenoidal projection Q, fp64.  Oracle -- test infrastructure only.

Eq. KKTPO replaces the multiplier of div v* = 0 by the projection Q; the paper
computes it with a multigrid Poisson solve (Sec. 4.1).  The oracle uses the
definition itself: Q v = v - G phi with (D G) phi = D v on the closed box
(Neumann Laplacian), solved exactly by a sparse factorisation with one cell
grounded (the constant is the Laplacian's null space and G removes it).
"""

import numpy as np
import scipy.sparse.linalg as spla

from . import mac


_FACTORS = {}


def _factor(grid):
    key = grid.key()
    if key not in _FACTORS:
        o = mac.ops(grid)
        L = (o["D"] @ o["G"]).tocsc()
        _FACTORS[key] = spla.factorized(L[1:, 1:].tocsc())
    return _FACTORS[key]


def poisson_neumann(grid, b):
    """Solve (D G) phi = b (b must have zero mean); returns the mean-zero phi."""
    solve = _factor(grid)
    phi = np.zeros(grid.C)
    phi[1:] = solve(b[1:])
    return phi - phi.mean()


def project(grid, v):
    """Q v: the divergence-free part of v (wall faces stay zero)."""
    o = mac.ops(grid)
    v = v * o["mask"]
    phi = poisson_neumann(grid, o["D"] @ v)
    return v - o["G"] @ phi
