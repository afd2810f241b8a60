"""AO fixed-point iteration (Alg. 1) and the ADMM outer loop (Alg. 3), fp64.
Oracle -- test infrastructure only.

Readings:
* v_0 is fixed (given); so is v*_0 = v_0, and lambda_0 stays 0.
* Alg. 1 sets v* = v + lambda/K; its forward/backward pair is then repeated
  ``ao_iters`` times (Table 2: 2 iterations).  The initialisation is done at
  the first ADMM iteration only: later ADMM iterations continue the AO
  fixed-point iteration from the previous v* (warm start).  With a fixed,
  small number of AO passes, re-initialising at w = v + lambda/K every time
  biases the ADMM fixed point away from the KKT point (the AO gradient is then
  taken at w, not at v*): on an 8^2 x 4 problem the relative KKT residual
  stalled at 0.09 that way, and keeps falling with the warm start.
* Alg. 3's inner loop runs at least one V-cycle per ADMM iteration, so that v
  follows every new target; then V-cycles until ||f||_inf <= eps * ||f||_inf
  of the first NSO.
* the backward sweep is the exact adjoint of the forward sweep that preceded
  it: every A(v*_i) and Taylor order K_i in it is the one the forward sweep
  used; the new v* replaces the old only once the sweep is done.
* NSO target z_i = v*_i - lambda_i / K (scaled ADMM form of Eq. optAdmm).
* stopping: the relative KKT residual R(v) = ||g(v)|| / ||g(v_start)|| <= tol,
  or Alg. 3's max_i ||rho_i^last - rho_i||_inf < eps_admm.
"""
import numpy as np

from . import kkt, projection, stfas


def ao(P, v, lam, iters=None, start=None):
    """Alg. 1.  Returns (v*, rhos, Ks) -- rhos/Ks from the last forward sweep.

    ``start``: the v* to continue from (warm start); None initialises v* = w."""
    iters = P.ao_iters if iters is None else iters
    N = P.N
    w = v[:N] + lam / P.K
    w[0] = P.v0
    vstar = w.copy() if start is None else start.copy()
    for _ in range(iters):
        rhos, Ks = kkt.forward_density(P, vstar)
        mu = kkt.adjoint_density(P, vstar, rhos, Ks)
        dens = kkt.density_gradient(P, vstar, rhos, Ks, mu)   # -(dA/dv*)^T mu
        new = vstar.copy()
        for i in range(1, N):
            new[i] = projection.project(P.grid, w[i] - dens[i] / P.K)
        vstar = new
    return vstar, rhos, Ks


def ao_objective(P, w, vstar):
    rhos, _ = kkt.forward_density(P, vstar)
    d = (w - vstar)[1:]
    return P.misfit(rhos) + 0.5 * P.K * float(np.sum(d * d))


def nso(P, x, z, fscale, eps_rel, max_cycles):
    """Alg. 3 inner loop: at least one V-cycle, then V-cycles until
    ||f||_inf <= eps_rel * fscale (or the cap)."""
    f = kkt.state_inf(kkt.nso_residual(P, P.grid, x, z))
    cycles = 0
    while (cycles < 1 or f > eps_rel * fscale) and cycles < max_cycles:
        f = stfas.stfas_cycle(P, x, z)
        cycles += 1
    return f, cycles


def solve(P, tol=1e-6, max_admm=50, eps_admm=None, eps_stfas=1e-5, max_vcycles=20,
          callback=None):
    """Alg. 3 with the stopping readings above.  Returns (x, vstar, lam, history)."""
    N = P.N
    if eps_admm is None:
        eps_admm = P.rho_scale / 100.0
    v = np.zeros((N + 1, P.grid.F))
    v[0] = P.v0
    lam = np.zeros((N, P.grid.F))
    x = kkt.zero_state(P)
    x["v"] = v
    rho_last, _ = kkt.forward_density(P, v)
    g0 = kkt.kkt_norm(P, v)
    hist = []
    fscale = None
    vstar = None
    for it in range(max_admm):
        vstar, rhos, _ = ao(P, x["v"], lam, start=vstar)
        z = vstar - lam / P.K
        if fscale is None:
            fscale = kkt.state_inf(kkt.nso_residual(P, P.grid, x, z))
        fres, cycles = nso(P, x, z, fscale, eps_stfas, max_vcycles)
        R = kkt.kkt_norm(P, x["v"]) / g0
        dr = float(np.max(np.abs(rho_last - rhos)))
        hist.append(dict(it=it, kkt_rel=R, f_inf=fres, vcycles=cycles, drho=dr,
                         objective=kkt.objective(P, x["v"])))
        if callback:
            callback(hist[-1])
        if R <= tol or dr < eps_admm:
            break
        rho_last = rhos
        lam[1:N] += P.K * P.beta * (x["v"][1:N] - vstar[1:N])
    return x, vstar, lam, hist
