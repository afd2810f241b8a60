"""Writes autograd_32cubed.npz: the fp64 oracle's loss and gradient of the
differentiable forward simulation at 32^3 (the reference of the GPU test of
the torch.autograd.Function at that size).  Calls only oracle/ and the input
generators.

Problem: the differentiable-simulation recipe (workloads.config_autograd) at
32^3 cells and 2 steps of dt = 1/48 (the step of the 128^3 x 48 workload):
Gaussian ball rho_0, seeded smooth random forces (correlation length 8
cells, max |u| = 0.1), loss 1/2 ||rho_N - rho*||^2 to a blurred ellipsoid
union.  The oracle solves each implicit step exactly (Newton on the saddle
system, sparse direct solves) and differentiates the chain by its adjoint
(brute.objective_and_gradient).  Stored: the loss, ||g||, and the gradient's
projections on 32 seeded random directions (workloads.random_faces3 with
seeds 9000..9031), so a changed term shows up without storing the whole
field.  Takes about half an hour on one core.

Run from the repository root: python tests/golden/make_autograd_32.py
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import brute, kkt  # noqa: E402
from paper_1608_01102_gb300 import workloads  # noqa: E402

N_DIRS = 32


def case():
    n, N = 32, 2
    cfg = workloads.config_autograd(n, N)
    P = kkt.Problem(n, n, N, 1.0 / 48, cfg["rho0"], r=1e-30, K=1.0, keyframes={N: (cfg["star"], 1.0)},
                    metric_levels=0, nz=n)
    return P, cfg["u"] * P.grid.interior_faces()


def directions(P):
    return [np.random.default_rng(9000 + k).standard_normal((P.N, P.grid.F)) * P.grid.interior_faces()
            for k in range(N_DIRS)]


def main():
    P, u = case()
    J, g = brute.objective_and_gradient(P, u)
    proj = np.array([float(np.sum(g * d)) for d in directions(P)])
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "autograd_32cubed.npz")
    np.savez(out, loss=J, gnorm=float(np.linalg.norm(g)), proj=proj)
    print(out, J, np.linalg.norm(g))


if __name__ == "__main__":
    main()
