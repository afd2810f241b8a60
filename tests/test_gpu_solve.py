"""Whole solves on the GPU against the fp64 oracle at a matched KKT residual.

The reference is tests/golden/admm_solved_8x8x4.npz, written by
tests/golden/make_admm_solved.py (the oracle's Alg. 3 with residual balancing
of K, solved to a relative KKT residual of 1e-7).  The library solves the same
problem from v = 0 with the same rule; the precision policy's tolerances apply to the
result: force field relative L2 <= 1e-3 and objective relative <= 1e-4.
"""
import os

import numpy as np
import pytest

from oracle import kkt
from paper_1608_01102_gb300 import stc, workloads

from gpu_common import rel

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "admm_solved_8x8x4.npz")


def _problem():
    n, N = 8, 4
    rho0 = workloads.gaussian_ball(n, n, (0.5, 0.35), 0.15)
    star = workloads.gaussian_ball(n, n, (0.5, 0.65), 0.15)
    P = kkt.Problem(n, n, N, 1.0 / N, rho0, r=1e-2, K=1.0, keyframes={N: (star, 1.0)}, metric_levels=0)
    return P, rho0, star


@pytest.mark.parametrize("prec,tol", [(1, 1e-7), (0, 1e-4)])
def test_solve_matches_the_oracle_at_a_matched_kkt_residual(prec, tol):
    ref = np.load(GOLDEN)
    assert ref["kkt_rel"] <= 1e-7
    P, rho0, star = _problem()
    N = P.N
    prm = stc.default_params(8, 8, N, precision=prec, r=1e-2, K=1.0, metric_levels=0, eps_admm=0.0, k_adapt=1)
    with stc.Problem(prm, rho0) as G:
        G.set_keyframes({N: (star, 1.0)})
        rep = G.solve(tol=tol, max_admm=600)
        assert rep["kkt_rel"] <= tol, rep
        v = G.get("V")
        G.kkt_residual()
        u = G.get("KKT_U")
    # the objective of Eq. opt, evaluated by the oracle on the GPU's v
    J = kkt.objective(P, v)
    assert abs(J - float(ref["objective"])) <= 1e-4 * float(ref["objective"]), (J, float(ref["objective"]))
    assert abs(rep["objective"] - float(ref["objective"])) <= 1e-4 * float(ref["objective"])
    assert rel(u, ref["u"]) <= 1e-3, rel(u, ref["u"])
    assert rel(u, kkt.forces(P, v)) <= (1e-10 if prec else 2e-5)
