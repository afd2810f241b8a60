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
* Sec. 5 (convergence analysis) safeguards Alg. 1 by blending: the fixed-point
  update y = Q(w - dPhi/K) is not taken whole; v* moves to v* + a (y - v*) with
  a = 1, 1/2, 1/4, ... until the AO objective (Eq. PO) does not increase.  The
  blend of two solenoidal fields is solenoidal, so no projection follows it.
  ``P.ao_halvings`` bounds the halvings (default 8); when none of the trials
  decreases the objective, v* is kept and the remaining AO passes are skipped
  (they would repeat the same trials).  A trial whose Taylor series does not
  reach the tolerance within taylor_kmax counts as rejected.  Descent along
  y - v* is guaranteed only for solenoidal w (as in Alg. 3, where v and lambda
  are solenoidal); ``ao_halvings = -1`` is the plain Alg. 1
  (a = 1 always).  Without the blend, K = 1 on 32^2 x 16 sent the AO objective
  up and down between ADMM iterations and the relative KKT residual climbed to
  15; with it the same run falls below 1 within 20 iterations.
* ao() returns the densities and Taylor orders of a forward sweep at the
  final v* (the blend evaluates them anyway; the plain form runs one more sweep).
* Alg. 3's inner loop runs at least one V-cycle per ADMM iteration, so that v
  follows every new target; then V-cycles until ||f||_inf <= eps * ||f||_inf
  of the first NSO.
* the backward sweep is the exact adjoint of the forward sweep that preceded
  it: every A(v*_i) and Taylor order K_i in it is the one the forward sweep
  used; the new v* replaces the old only once the sweep is done.
* NSO target z_i = v*_i - lambda_i / K (scaled ADMM form of Eq. optAdmm).
* stopping: the relative KKT residual R(v) = ||g(v)|| / ||g(v_start)|| <= tol,
  or Alg. 3's max_i ||rho_i^last - rho_i||_inf < eps_admm.
* residual balancing of the penalty (``P.k_adapt``, off by default: Alg. 3
  keeps Table 2's constant K; an extension, not the paper's): after each
  multiplier update, with the primal residual r_p = ||v - v*|| and the dual
  residual r_d = K ||v - v_prev|| over steps 1..N-1 (v_prev: v at the
  previous update), K doubles when r_p > 10 r_d and halves when r_d > 10 r_p,
  within 2^+-10 of its starting value.  The fixed point of the iteration does
  not depend on K (Sec. 4: K sets the rate); the target z and the AO centre w
  use the new K through the unscaled multiplier.
* Sec. 5's augmented-Lagrangian fallback (``P.al_threshold`` >= 0; default -1
  = the plain Alg. 3): the multiplier update is applied only once the
  objective J(v) of Eq. opt stops decreasing by more than al_threshold * |J|
  between ADMM iterations (the first iteration compares with J(v_start));
  otherwise the AO/NSO alternation continues with the same lambda.
"""
import numpy as np

from . import advection, kkt, projection, stfas

LM_MAX_RATIO = 4.0 ** 6   # largest LM shift relative to its default
ADAPT_MU, ADAPT_TAU, ADAPT_RANGE = 10.0, 2.0, 1024.0   # residual balancing of K (P.k_adapt)


def ao(P, v, lam, iters=None, start=None, trace=None):
    """Alg. 1 with Sec. 5's blending safeguard.  Returns (v*, rhos, Ks) with
    rhos/Ks from a forward sweep at the returned v*.

    ``start``: the v* to continue from (warm start); None initialises v* = w.
    ``trace``: a list that receives, per AO pass, the number of halvings taken
    (-1 when every trial was rejected)."""
    iters = P.ao_iters if iters is None else iters
    N = P.N
    w = v[:N] + lam / P.K
    w[0] = P.v0
    vstar = w.copy() if start is None else start.copy()
    rhos, Ks = kkt.forward_density(P, vstar)
    J = ao_objective_from(P, w, vstar, rhos)
    for _ in range(iters):
        mu = kkt.adjoint_density(P, vstar, rhos, Ks)
        dens = kkt.density_gradient(P, vstar, rhos, Ks, mu)   # -(dA/dv*)^T mu
        y = vstar.copy()
        for i in range(1, N):
            y[i] = projection.project(P.grid, w[i] - dens[i] / P.K)
        if P.ao_halvings < 0:                  # plain Alg. 1
            vstar = y
            rhos, Ks = kkt.forward_density(P, vstar)
            J = ao_objective_from(P, w, vstar, rhos)
            if trace is not None:
                trace.append(0)
            continue
        a, taken = 1.0, -1
        for h in range(P.ao_halvings + 1):
            cand = vstar + a * (y - vstar)
            try:
                rc, kc = kkt.forward_density(P, cand)
                Jc = ao_objective_from(P, w, cand, rc)
            except advection.TaylorOrderError:
                Jc = np.inf                    # a trial too fast to advect is rejected
            if Jc <= J:
                vstar, rhos, Ks, J, taken = cand, rc, kc, Jc, h
                break
            a *= 0.5
        if trace is not None:
            trace.append(taken)
        if taken < 0:
            break
    return vstar, rhos, Ks


def ao_objective_from(P, w, vstar, rhos):
    """Eq. PO's objective: keyframe misfit in the C_i metric plus
    K/2 sum_{i=1}^{N-1} ||w_i - v*_i||^2 (v*_0 = v_0 is fixed)."""
    d = (w - vstar)[1:]
    return P.misfit(rhos) + 0.5 * P.K * float(np.sum(d * d))


def ao_objective(P, w, vstar):
    rhos, _ = kkt.forward_density(P, vstar)
    return ao_objective_from(P, w, vstar, rhos)


def nso(P, x, z, fscale, eps_rel, max_cycles, lm=None):
    """Alg. 3 inner loop: at least one V-cycle, then V-cycles until
    ||f||_inf <= eps_rel * fscale (or the cap).

    ``lm`` (a dict with "gamma", "gamma0", "rejected"; used when P.lm_adapt):
    Sec. 5's Levenberg-Marquardt safeguard -- the FAS cycle acts as the
    subproblem solver of an LM method whose damping is the shift gamma of the
    smoother's v blocks.  A cycle that raises ||f||_inf (or fails: a
    non-finite norm, a singular local solve) is undone and gamma quadrupled;
    gamma does not fall during one NSO solve and is halved back toward its
    default when the next one starts (halving after each accepted cycle made
    gamma oscillate: every third cycle was undone on rough targets).  gamma
    stays below LM_MAX_RATIO times its default; a cycle undone at that bound
    ends the solve (unbounded growth left every later cycle undone).  f
    itself, and so the fixed point, does not depend on gamma.  Returns
    (||f||_inf, cycles)."""
    if lm is not None and P.lm_adapt:
        lm["gamma"] = max(lm["gamma0"], 0.5 * lm["gamma"])
    f = kkt.state_inf(kkt.nso_residual(P, P.grid, x, z))
    cycles = 0
    while (cycles < 1 or f > eps_rel * fscale) and cycles < max_cycles:
        cycles += 1
        if lm is None or not P.lm_adapt:
            f = stfas.stfas_cycle(P, x, z)
            continue
        keep = kkt.copy_state(x)
        P.lm_shift = lm["gamma"]
        try:
            fn = stfas.stfas_cycle(P, x, z)
        except np.linalg.LinAlgError:
            fn = np.inf
        if fn <= f:
            f = fn
        else:
            for k in x:
                x[k] = keep[k]
            lm["rejected"] += 1
            if lm["gamma"] >= LM_MAX_RATIO * lm["gamma0"]:
                break                          # undone even at the largest shift: give up this solve
            lm["gamma"] = min(4.0 * lm["gamma"], LM_MAX_RATIO * lm["gamma0"])
    if lm is not None:
        P.lm_shift = lm["gamma"]
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
    J_prev = kkt.objective(P, v)
    updates = 0
    hist = []
    fscale = None
    vstar = None
    lm = dict(gamma=P.lm_shift, gamma0=P.lm_shift, rejected=0)
    K0 = P.K
    v_prev = None
    for it in range(max_admm):
        vstar, rhos, _ = ao(P, x["v"], lam, start=vstar)
        z = vstar - lam / P.K
        if fscale is None:
            fscale = kkt.state_inf(kkt.nso_residual(P, P.grid, x, z))
        fres, cycles = nso(P, x, z, fscale, eps_stfas, max_vcycles, lm)
        R = kkt.kkt_norm(P, x["v"]) / g0
        dr = float(np.max(np.abs(rho_last - rhos)))
        J = kkt.objective(P, x["v"])
        apply = P.al_threshold < 0 or (J_prev - J) <= P.al_threshold * abs(J_prev)
        hist.append(dict(it=it, kkt_rel=R, f_inf=fres, vcycles=cycles, drho=dr,
                         objective=J, rejected=lm["rejected"], lm_shift=lm["gamma"],
                         lambda_updates=updates + (1 if apply else 0), K=P.K))
        J_prev = J
        if callback:
            callback(hist[-1])
        if R <= tol or dr < eps_admm:
            break
        rho_last = rhos
        if apply:
            lam[1:N] += P.K * P.beta * (x["v"][1:N] - vstar[1:N])
            updates += 1
            if P.k_adapt:
                if v_prev is not None and N > 1:
                    rp = float(np.linalg.norm(x["v"][1:N] - vstar[1:N]))
                    rd = P.K * float(np.linalg.norm(x["v"][1:N] - v_prev[1:N]))
                    hist[-1]["r_primal"], hist[-1]["r_dual"] = rp, rd
                    Kn = P.K
                    if rp > ADAPT_MU * rd:
                        Kn = P.K * ADAPT_TAU
                    elif rd > ADAPT_MU * rp:
                        Kn = P.K / ADAPT_TAU
                    P.K = min(max(Kn, K0 / ADAPT_RANGE), K0 * ADAPT_RANGE)
                v_prev = x["v"].copy()
    P.lm_shift = lm["gamma0"]
    P.K = K0
    return x, vstar, lam, hist
