"""Writes admm_solved_8x8x4.npz: the fp64 oracle's ADMM solve (Alg. 3 with
residual balancing of K) of a tiny problem to a relative KKT residual of 1e-7,
the reference of the matched-residual GPU test (forces and objective at the
same residual).  Calls only oracle/ and the input generators.

Problem: 8^2 cells, N = 4, dt = 1/4, Gaussian ball (sigma 0.15) from (0.5,
0.35) to a keyframe at (0.5, 0.65) at t = T, r = 1e-2, C_i = I, K = 1.

Run from the repository root: python tests/golden/make_admm_solved.py
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import admm, kkt  # noqa: E402
from paper_1608_01102_gb300 import workloads  # noqa: E402


def problem():
    n, N = 8, 4
    rho0 = workloads.gaussian_ball(n, n, (0.5, 0.35), 0.15)
    star = workloads.gaussian_ball(n, n, (0.5, 0.65), 0.15)
    return kkt.Problem(n, n, N, 1.0 / N, rho0, r=1e-2, K=1.0, keyframes={N: (star, 1.0)}, metric_levels=0,
                       k_adapt=True)


def main():
    P = problem()
    x, vstar, lam, hist = admm.solve(P, tol=1e-7, max_admm=400, eps_admm=0.0)
    v = x["v"]
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "admm_solved_8x8x4.npz")
    np.savez(out, v=v, u=kkt.forces(P, v), objective=kkt.objective(P, v), kkt_rel=hist[-1]["kkt_rel"],
             iters=len(hist), kkt_history=np.array([h["kkt_rel"] for h in hist]))
    print(out, len(hist), hist[-1]["kkt_rel"], kkt.objective(P, v))


if __name__ == "__main__":
    main()
