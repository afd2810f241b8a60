"""Problem statement, reduced objective / gradient, relative KKT residual and the
NSO residual f, fp64.  Oracle -- test infrastructure only.

Index conventions (Sec. 3): v_i, pbar_i for i = 0..N (v_0 is given and fixed),
u_i for i = 0..N-1, p_{i+1} for i = 0..N-1 (stored as p[i]), rho_i for
i = 0..N, adjoint mu_i for i = 0..N-1 (mu_N = 0, Eq. KKTPO).
"""
from dataclasses import dataclass, field

import numpy as np

from . import advection, mac, metric, projection


@dataclass
class Problem:
    nx: int
    ny: int
    N: int
    dt: float
    rho0: np.ndarray                 # (C,)
    r: float = 1e-3                  # force regularisation (Eq. opt)
    K: float = 10.0                  # ADMM penalty (Eq. optAdmm)
    beta: float = 1.0                # multiplier step (Alg. 3)
    v0: np.ndarray = None            # (F,) fixed initial velocity, default 0
    keyframes: dict = field(default_factory=dict)   # step -> (rho_star (C,), c_i)
    metric_levels: int = 0
    metric_sigma0: float = 1.0
    taylor_tol: float = 1e-5
    taylor_kmax: int = 64
    ao_iters: int = 2
    ao_halvings: int = 8             # Sec. 5 blending safeguard of Alg. 1 (-1: plain)
    pre: int = 2
    post: int = 2
    coarse_sweeps: int = 10
    coarsest_n: int = 4
    omega: float = 0.8               # SCGS under-relaxation
    cgc_guard: bool = True           # keep a coarse correction only if it lowers ||res - f||_2
    lm_adapt: bool = True            # Sec. 5 LM safeguard of the NSO loop (adaptive lm_shift)
    al_threshold: float = -1.0       # Sec. 5 AL fallback: lambda update only when J stalls (<0: off)
    time_coarsen: bool = False       # STFAS coarse levels halve N too (the paper: space only)
    self_advection: bool = True      # False drops Adv (linear saddle problem; pins only)
    lm_shift: float = None           # LM shift of the smoother's v blocks, default 1/dt^2
    nz: int = 0                      # 0: the 2D grid nx x ny; > 0: the 3D grid nx x ny x nz
    periodic: bool = False           # 3D only: every axis wraps (the paper's periodic benchmarks)
    k_adapt: bool = False            # residual balancing of the ADMM penalty K in solve() (not in the paper)

    def __post_init__(self):
        self.h = 1.0 / self.nx
        if self.periodic and not self.nz:
            raise ValueError("periodic boundaries are built for the 3D grid")
        self.grid = (mac.Grid3(self.nx, self.ny, self.nz, self.h, self.periodic) if self.nz
                     else mac.Grid(self.nx, self.ny, self.h))
        self.rho0 = np.asarray(self.rho0, float).ravel()
        if self.v0 is None:
            self.v0 = np.zeros(self.grid.F)
        self.rho_scale = float(np.max(np.abs(self.rho0)))
        if self.lm_shift is None:
            self.lm_shift = 1.0 / (self.dt * self.dt)

    # keyframe metric terms --------------------------------------------------
    def misfit_grad(self, i, rho_i):
        """C_i (rho_i - rho*_i), zero where step i has no keyframe."""
        if i not in self.keyframes:
            return np.zeros(self.grid.C)
        star, c = self.keyframes[i]
        return metric.apply_metric(self.nx, self.ny, rho_i - star, self.metric_levels,
                                   self.metric_sigma0, c, self.nz, self.periodic)

    def misfit(self, rhos):
        e = 0.0
        for i in self.keyframes:
            star, _ = self.keyframes[i]
            e += 0.5 * float((rhos[i] - star) @ self.misfit_grad(i, rhos[i]))
        return e


# ---------------------------------------------------------------------------
# Density forward / adjoint sweeps (Eq. Conv, Eq. KKTPO)
# ---------------------------------------------------------------------------

def forward_density(P, v, Ks=None):
    """rho_{i+1} = A[rho_i, v_i] for i = 0..N-1; returns (rhos (N+1, C), Ks (N,)).

    With ``Ks`` given the Taylor orders are frozen (finite-difference pins)."""
    rhos = [P.rho0.copy()]
    out = []
    for i in range(P.N):
        if Ks is None:
            nxt, k, _ = advection.taylor_forward(P.grid, v[i], rhos[-1], P.dt, P.taylor_tol,
                                                 P.rho_scale, P.taylor_kmax)
        else:
            k = int(Ks[i])
            nxt = advection.taylor_apply(P.grid, v[i], rhos[-1], P.dt, k)
        rhos.append(nxt)
        out.append(k)
    return np.array(rhos), np.array(out)


def adjoint_density(P, v, rhos, Ks):
    """mu_{i-1} = (dA[rho_i, v_i]/drho_i)^T mu_i - C_i (rho_i - rho*_i), i = N..1, mu_N = 0."""
    mu = np.zeros((P.N, P.grid.C))
    nxt = np.zeros(P.grid.C)   # mu_N
    for i in range(P.N, 0, -1):
        term = -P.misfit_grad(i, rhos[i])
        if i < P.N:
            term = term + advection.taylor_adjoint_rho(P.grid, v[i], nxt, P.dt, Ks[i])
        mu[i - 1] = term
        nxt = mu[i - 1]
    return mu


def density_gradient(P, v, rhos, Ks, mu):
    """d/dv_i of the density misfit = -(dA[rho_i, v_i]/dv_i)^T mu_i, i = 0..N-1."""
    out = np.zeros((P.N + 1, P.grid.F))
    for i in range(P.N):
        out[i] = -advection.taylor_adjoint_v(P.grid, v[i], rhos[i], mu[i], P.dt, Ks[i])
    return out


# ---------------------------------------------------------------------------
# Reduced problem in v (Appendix A: u eliminated) and the KKT metric
# ---------------------------------------------------------------------------

def forces(P, v):
    """u_i(v) = Q[(v_{i+1} - v_i)/dt + Adv(v_{i+1})], i = 0..N-1 (Appendix A)."""
    g = P.grid
    return np.array([projection.project(g, (v[i + 1] - v[i]) / P.dt + mac.adv(g, v[i + 1]))
                     for i in range(P.N)])


def objective(P, v, Ks=None):
    """J(v) = r/2 sum ||u_i(v)||^2 + 1/2 sum ||rho_i(v) - rho*_i||^2_{C_i} (Eq. opt)."""
    u = forces(P, v)
    rhos, _ = forward_density(P, v, Ks)
    return 0.5 * P.r * float(np.sum(u * u)) + P.misfit(rhos)


def reduced_gradient(P, v):
    """g_i = Q[ r(-u_i/dt + (I/dt + dAdv(v_i))^T u_{i-1}) - (dA[rho_i,v_i]/dv_i)^T mu_i ],
    i = 1..N (v_0 fixed: g_0 = 0; the u_N and mu_N terms vanish at i = N)."""
    g = P.grid
    u = forces(P, v)
    rhos, Ks = forward_density(P, v)
    mu = adjoint_density(P, v, rhos, Ks)
    dens = density_gradient(P, v, rhos, Ks, mu)
    out = np.zeros((P.N + 1, g.F))
    for i in range(1, P.N + 1):
        t = mac.adv_jacobian_T_apply(g, v[i], u[i - 1]) + u[i - 1] / P.dt
        if i < P.N:
            t = t - u[i] / P.dt
        t = P.r * t + dens[i]
        out[i] = projection.project(g, t)
    return out


def kkt_norm(P, v):
    return float(np.linalg.norm(reduced_gradient(P, v)))


# ---------------------------------------------------------------------------
# NSO residual f (Eq. KKTAO, Appendix A) and its potential
# ---------------------------------------------------------------------------

def zero_state(P, grid=None):
    g = grid or P.grid
    return dict(v=np.zeros((P.N + 1, g.F)), pbar=np.zeros((P.N + 1, g.C)),
                u=np.zeros((P.N, g.F)), p=np.zeros((P.N, g.C)))


def copy_state(x):
    return {k: a.copy() for k, a in x.items()}


def nso_residual(P, grid, x, z):
    """f(v, pbar, u, p) with the readings: v_0 fixed (its rows dropped), no K/r
    term at i = N, target z_i = v*_i - lambda_i/K.

    row 1, faces, i = 1..N : (K/r)(v_i - z_i)[i<N] - u_i/dt [i<N]
                             + (I/dt + dAdv(v_i))^T u_{i-1} + grad pbar_i
    row 2, cells, i = 1..N : -div v_i
    row 3, faces, i = 0..N-1: (v_{i+1} - v_i)/dt + Adv(v_{i+1}) - u_i + grad p_{i+1}
    row 4, cells, i = 0..N-1: -div u_i
    Wall-face rows are zero.
    """
    o = mac.ops(grid)
    N, dt, a = P.N, P.dt, P.K / P.r
    v, pb, u, p = x["v"], x["pbar"], x["u"], x["p"]
    f1 = np.zeros_like(v)
    f2 = np.zeros_like(pb)
    f3 = np.zeros_like(u)
    f4 = np.zeros_like(p)
    sa = 1.0 if P.self_advection else 0.0
    for i in range(1, N + 1):
        t = sa * mac.adv_jacobian_T_apply(grid, v[i], u[i - 1]) + u[i - 1] / dt + o["G"] @ pb[i]
        if i < N:
            t = t + a * (v[i] - z[i]) - u[i] / dt
        f1[i] = t * o["mask"]
        f2[i] = -(o["D"] @ v[i])
    for i in range(N):
        t = (v[i + 1] - v[i]) / dt + sa * mac.adv(grid, v[i + 1]) - u[i] + o["G"] @ p[i]
        f3[i] = t * o["mask"]
        f4[i] = -(o["D"] @ u[i])
    return dict(v=f1, pbar=f2, u=f3, p=f4)


def nso_potential(P, grid, x, z):
    """Phi with grad Phi = f (so the Jacobian of f is symmetric, Eq. HESS):
    Phi = (K/2r) sum_{i=1}^{N-1} ||v_i - z_i||^2 - 1/2 sum ||u_i||^2
          + sum u_i . ((v_{i+1} - v_i)/dt + Adv(v_{i+1}))
          - sum p_{i+1} . div u_i - sum_{i>=1} pbar_i . div v_i
    (all on interior faces)."""
    o = mac.ops(grid)
    m = o["mask"]
    N, dt, a = P.N, P.dt, P.K / P.r
    v = x["v"] * m
    u = x["u"] * m
    val = 0.0
    for i in range(1, N):
        d = v[i] - z[i] * m
        val += 0.5 * a * float(d @ d)
    for i in range(N):
        val += -0.5 * float(u[i] @ u[i])
        sa = 1.0 if P.self_advection else 0.0
        val += float(u[i] @ ((v[i + 1] - v[i]) / dt + sa * mac.adv(grid, v[i + 1])))
        val -= float(x["p"][i] @ (o["D"] @ u[i]))
    for i in range(1, N + 1):
        val -= float(x["pbar"][i] @ (o["D"] @ v[i]))
    return val


def state_sub(a, b):
    return {k: a[k] - b[k] for k in a}


def state_inf(r):
    return max(float(np.max(np.abs(r[k]))) for k in r)
