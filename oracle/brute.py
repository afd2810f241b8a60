"""Full-resimulation gradient-based reference solver for tiny grids, fp64.
Oracle -- test infrastructure only.

This is the comparison system of Sec. 5 (a quasi-Newton optimiser, history 8,
whose every gradient runs a forward fluid simulation and its adjoint).  The
control is u; each step solves the implicit Navier-Stokes step of Eq. NSA/NSB
exactly (Newton on the saddle system, sparse direct solves), the density is
advected with v_i (Eq. Conv), and the gradient comes from the adjoint of the
whole chain.  Used only to check that STFAS + ADMM reach the same objective.
"""
import numpy as np
import scipy.optimize as so
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import advection, kkt, mac


def _saddle(grid, A_int, o, idx):
    G = o["G"][idx][:, 1:]                 # ground cell 0
    return sp.bmat([[A_int, G], [G.T, None]]).tocsc()


def ns_step(grid, v_prev, u, dt, tol=1e-13, maxit=50):
    """Solve (v - v_prev)/dt + Adv(v) - u + grad p = 0, div v = 0 by Newton."""
    o = mac.ops(grid)
    idx = np.nonzero(o["mask"])[0]
    n = idx.size
    v = v_prev.copy()
    p = np.zeros(grid.C)
    for _ in range(maxit):
        R1 = ((v - v_prev) / dt + mac.adv(grid, v) - u + o["G"] @ p)[idx]
        R2 = -(o["D"] @ v)[1:]
        if max(np.max(np.abs(R1)), np.max(np.abs(R2)) if R2.size else 0.0) < tol:
            return v, p
        A = (sp.eye(grid.F) / dt + mac.adv_jacobian(grid, v)).tocsr()[idx][:, idx]
        M = _saddle(grid, A, o, idx)
        d = spla.spsolve(M, -np.concatenate([R1, R2]))
        v[idx] += d[:n]
        p[1:] += d[n:]
    raise RuntimeError("implicit Navier-Stokes step did not converge")


def ns_step_adjoint(grid, v_next, y, dt):
    """Pi^T y, Pi the solution operator of the linearised step at v_next."""
    o = mac.ops(grid)
    idx = np.nonzero(o["mask"])[0]
    A = (sp.eye(grid.F) / dt + mac.adv_jacobian(grid, v_next)).tocsr()[idx][:, idx]
    M = _saddle(grid, A.T.tocsr(), o, idx)
    rhs = np.concatenate([y[idx], np.zeros(grid.C - 1)])
    sol = spla.spsolve(M, rhs)
    out = np.zeros(grid.F)
    out[idx] = sol[:idx.size]
    return out


def simulate(P, u):
    v = np.zeros((P.N + 1, P.grid.F))
    v[0] = P.v0
    for i in range(P.N):
        v[i + 1], _ = ns_step(P.grid, v[i], u[i], P.dt)
    return v


def objective_and_gradient(P, u):
    """J(u) = r/2 sum ||u_i||^2 + density misfit, and dJ/du by the adjoint chain."""
    v = simulate(P, u)
    rhos, Ks = kkt.forward_density(P, v)
    J = 0.5 * P.r * float(np.sum(u * u)) + P.misfit(rhos)
    mu = kkt.adjoint_density(P, v, rhos, Ks)
    dens = kkt.density_gradient(P, v, rhos, Ks, mu)
    grad = np.zeros_like(u)
    a = np.zeros(P.grid.F)          # total adjoint of v_N (v_N moves no density)
    for i in range(P.N - 1, -1, -1):
        xi = ns_step_adjoint(P.grid, v[i + 1], a, P.dt)
        grad[i] = P.r * u[i] + xi
        a = dens[i] + xi / P.dt
    m = mac.ops(P.grid)["mask"]
    return J, grad * m


def solve(P, u0=None, maxiter=500, gtol=1e-10):
    """L-BFGS (history 8) on the full-resimulation objective."""
    m = mac.ops(P.grid)["mask"]
    idx = np.nonzero(m)[0]
    shape = (P.N, P.grid.F)
    u0 = np.zeros(shape) if u0 is None else u0

    def fun(x):
        u = np.zeros(shape)
        u[:, idx] = x.reshape(P.N, idx.size)
        J, g = objective_and_gradient(P, u)
        return J, g[:, idx].ravel()

    res = so.minimize(fun, u0[:, idx].ravel(), jac=True, method="L-BFGS-B",
                      options=dict(maxcor=8, maxiter=maxiter, gtol=gtol, ftol=1e-15))
    u = np.zeros(shape)
    u[:, idx] = res.x.reshape(P.N, idx.size)
    return u, res
