"""Shared helpers of the GPU parity tests: build the same problem for the CUDA
library (through the C ABI) and for the fp64 oracle from one seeded recipe."""
import numpy as np

from oracle import kkt
from paper_1608_01102_gb300 import stc, workloads

# tolerances (relative L2 unless stated):
#  fp64 mode: the same arithmetic up to summation order (and the multigrid
#  projection's truncation, ~1e-8 after 8 cycles); fp32 mode: the bounds of the
#  precision policy -- per-step density 1e-5, state of one smoothing sweep or
#  V-cycle 1e-4 (fp32 epsilon times the conditioning of the saddle blocks,
#  K/r + 1/dt^2 ~ 1e3..1e4).
TOL = {1: dict(exact=1e-10, smooth=1e-8, project=2e-7, vcycle=1e-7, ao=1e-6),
       0: dict(exact=2e-6, smooth=1e-4, project=2e-5, vcycle=2e-4, ao=2e-4)}


def rel(a, b, floor=1e-30):
    a = np.asarray(a, float)
    b = np.asarray(b, float)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), floor))


def make_pair(nx=16, ny=None, N=6, precision=1, levels=2, r=1e-2, K=1.0, keyframes="end", v0=None,
              sigma=0.12, dt=None, **over):
    ny = ny or nx
    rho0 = workloads.gaussian_ball(nx, ny, (0.5, 0.35 * ny / nx), sigma)
    star = workloads.gaussian_ball(nx, ny, (0.5, 0.65 * ny / nx), sigma)
    if keyframes == "end":
        kf = {N: (star, 1.0)}
    elif keyframes is None:
        kf = {}
    else:
        kf = keyframes
    gpu_only = ("poisson_vcycles", "scgs_omega", "ao_trials", "scgs_cta_cells")   # kernel / schedule choices
    o_over = {k: v for k, v in over.items() if k not in gpu_only}
    if "scgs_omega" in over:
        o_over["omega"] = over["scgs_omega"]
    dt = 1.0 / N if dt is None else dt
    P = kkt.Problem(nx, ny, N, dt, rho0, r=r, K=K, keyframes=kf, metric_levels=levels, **o_over)
    if v0 is not None:
        P.v0 = v0.copy()
    prm = stc.default_params(nx, ny, N, precision=precision, r=r, K=K, metric_levels=levels, dt=dt)
    for k, v in over.items():
        setattr(prm, k, int(v) if isinstance(v, bool) else v)
    G = stc.Problem(prm, rho0, v0)
    if kf:
        G.set_keyframes(kf)
    return P, G


def velocity_trajectory(nx, ny, N, amp=0.6, seed=0, noise=0.05):
    """A smooth swirl whose amplitude and centre drift with time, plus a little
    seeded noise (wall faces zero): N+1 face slabs, slab 0 = 0."""
    rng = np.random.default_rng(seed)
    m = workloads.interior_face_mask(nx, ny)
    v = np.zeros((N + 1, workloads.face_count(nx, ny)))
    for i in range(1, N + 1):
        c = (0.5 + 0.1 * np.sin(i), 0.5 + 0.1 * np.cos(i))
        v[i] = workloads.swirl_velocity(nx, ny, amp * (1 + 0.3 * np.sin(0.7 * i)), c, 0.25)
        v[i] += noise * amp * rng.standard_normal(v.shape[1]) * m
    return v


def random_state(P, seed, grid=None, scale=1.0):
    rng = np.random.default_rng(seed)
    g = grid or P.grid
    m = g.interior_faces()
    x = dict(v=rng.standard_normal((P.N + 1, g.F)) * m * scale,
             pbar=rng.standard_normal((P.N + 1, g.C)),
             u=rng.standard_normal((P.N, g.F)) * m,
             p=rng.standard_normal((P.N, g.C)))
    x["v"][0] = 0.0
    x["pbar"][0] = 0.0
    return x
