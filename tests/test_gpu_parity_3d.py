"""GPU parity on the 3D grid: every step of the hot path, called through the C
ABI of libstc, against the fp64 oracle (mac.Grid3) on the same seeded inputs.

Tolerances as the 2D tests (gpu_common.TOL).  Grids are non-cubic so that the
three axes' index arithmetic is exercised separately; each spans several
colour tiles.
"""
import numpy as np
import pytest

from oracle import admm, kkt, mac, projection, scgs, stfas
from paper_1608_01102_gb300 import stc, workloads

from gpu_common import TOL, rel

pytestmark = [pytest.mark.gpu, pytest.mark.filterwarnings("ignore::DeprecationWarning")]

PREC = [1, 0]


def make_pair3(nx, ny, nz, N, precision=1, levels=1, r=1e-2, K=1.0, keyframes="end", sigma=0.15, dt=None,
               periodic=False, **over):
    rho0 = workloads.gaussian_ball3(nx, ny, nz, (0.5, 0.35 * ny / nx, 0.5 * nz / nx), sigma)
    star = workloads.gaussian_ball3(nx, ny, nz, (0.5, 0.65 * ny / nx, 0.45 * nz / nx), sigma)
    kf = {N: (star, 1.0)} if keyframes == "end" else (keyframes or {})
    dt = 1.0 / N if dt is None else dt
    o_over = {k: v for k, v in over.items() if k not in ("poisson_vcycles", "scgs_omega")}
    P = kkt.Problem(nx, ny, N, dt, rho0, r=r, K=K, keyframes=kf, metric_levels=levels, nz=nz, periodic=periodic,
                    **o_over)
    prm = stc.default_params(nx, ny, N, precision=precision, r=r, K=K, metric_levels=levels, dt=dt, nz=nz,
                             boundary=1 if periodic else 0)
    for k, v in over.items():
        setattr(prm, k, int(v) if isinstance(v, bool) else v)
    G = stc.Problem(prm, rho0)
    if kf:
        G.set_keyframes(kf)
    return P, G


def velocity3(nx, ny, nz, N, amp=0.6, seed=0, noise=0.05, periodic=False):
    rng = np.random.default_rng(seed)
    m = workloads.interior_face_mask3(nx, ny, nz, periodic)
    v = np.zeros((N + 1, workloads.face_count3(nx, ny, nz)))
    for i in range(1, N + 1):
        c = (0.5 + 0.1 * np.sin(i), 0.5 * ny / nx + 0.05 * np.cos(i), 0.5 * nz / nx)
        v[i] = workloads.swirl_velocity3(nx, ny, nz, amp * (1 + 0.3 * np.sin(0.7 * i)), c, 0.3)
        v[i] += noise * amp * rng.standard_normal(v.shape[1]) * m
    return v


def random_state3(P, seed, grid=None, scale=1.0):
    rng = np.random.default_rng(seed)
    g = grid or P.grid
    m = g.interior_faces()
    x = dict(v=rng.standard_normal((P.N + 1, g.F)) * m * scale, pbar=rng.standard_normal((P.N + 1, g.C)),
             u=rng.standard_normal((P.N, g.F)) * m, p=rng.standard_normal((P.N, g.C)))
    x["v"][0] = 0.0
    x["pbar"][0] = 0.0
    return x


def test_level_dims_and_sizes():
    P, G = make_pair3(16, 8, 12, 2, precision=0, coarsest_n=2)
    grids = stfas.hierarchy(P)
    assert G.num_levels() == len(grids) == 3
    for l, g in enumerate(grids):
        assert G.level_shape(l) == (g.nx, g.ny, g.nz)
        assert G.field_shape("V", l) == (3, g.F) and G.field_shape("P", l) == (2, g.C)


# ---------------------------------------------------------------------------
# a2: projection (batched multigrid over the step's fields)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("prec", PREC)
@pytest.mark.parametrize("shape", [(8, 8, 8), (16, 8, 12), (12, 12, 8)])
def test_projection_3d(prec, shape):
    nx, ny, nz = shape
    P, G = make_pair3(nx, ny, nz, 3, precision=prec)
    rng = np.random.default_rng(1)
    w = workloads.random_faces3(rng, nx, ny, nz, 3)
    w[1] += workloads.swirl_velocity3(nx, ny, nz, 3.0)
    G.set("W", w)
    G.project("W", 0, 3)
    out = G.get("W")
    for i in range(3):
        ref = projection.project(P.grid, w[i])
        assert rel(out[i], ref) < TOL[prec]["project"] * 5, (i, rel(out[i], ref))


# ---------------------------------------------------------------------------
# a3: forward advection (Taylor exponential, adaptive order)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("prec", PREC)
@pytest.mark.parametrize("shape,N", [((12, 8, 10), 4), ((8, 8, 8), 5), ((16, 12, 6), 3)])
def test_forward_advection_3d(prec, shape, N):
    nx, ny, nz = shape
    P, G = make_pair3(nx, ny, nz, N, precision=prec)
    v = velocity3(nx, ny, nz, N, amp=0.8)
    G.set("VSTAR", v[:N])
    G.advect("VSTAR")
    rho = G.get("RHO")
    K = G.taylor_orders()
    ref, Kref = kkt.forward_density(P, v[:N])
    np.testing.assert_array_equal(K, Kref)
    assert max(Kref) > 2
    for i in range(N + 1):
        assert rel(rho[i], ref[i]) < (1e-12 if prec == 1 else 1e-5), (i, rel(rho[i], ref[i]))
    assert abs(rho[N].sum() - P.rho0.sum()) < (1e-10 if prec == 1 else 1e-4) * P.rho0.sum()


# ---------------------------------------------------------------------------
# a5 / a6 / a7: keyframe metric, backward adjoint sweep, v*-gradient
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("prec", PREC)
@pytest.mark.parametrize("shape,N,levels", [((12, 8, 10), 4, 1), ((8, 8, 8), 5, 2), ((16, 8, 8), 3, 0)])
def test_adjoint_sweep_3d(prec, shape, N, levels):
    nx, ny, nz = shape
    mid = workloads.gaussian_ball3(nx, ny, nz, (0.4, 0.5 * ny / nx, 0.5 * nz / nx), 0.12)
    end = workloads.gaussian_ball3(nx, ny, nz, (0.6, 0.6 * ny / nx, 0.4 * nz / nx), 0.12)
    kf = {N // 2: (mid, 0.5), N: (end, 1.0)}
    P, G = make_pair3(nx, ny, nz, N, precision=prec, levels=levels, keyframes=kf, K=2.0)
    v = velocity3(nx, ny, nz, N, amp=0.7, seed=3)
    w = workloads.random_faces3(np.random.default_rng(4), nx, ny, nz, N, 0.2)
    G.set("VSTAR", v[:N])
    G.set("W", w)
    G.advect("VSTAR")
    G.metric_terms()
    G.adjoint("VSTAR", 1.0, 1.0 / P.K)
    rhos, Ks = kkt.forward_density(P, v[:N])
    mt = G.get("MTERM")
    for s in range(N + 1):
        ref = P.misfit_grad(s, rhos[s])
        if s in kf:
            assert rel(mt[s], ref) < (1e-11 if prec == 1 else 2e-5), (s, rel(mt[s], ref))
        else:
            assert np.all(mt[s] == 0)
    mu = G.get("MU")
    mu_ref = kkt.adjoint_density(P, v[:N], rhos, Ks)
    for s in range(N):
        assert rel(mu[s], mu_ref[s]) < (1e-11 if prec == 1 else 2e-5), (s, rel(mu[s], mu_ref[s]))
    dens = kkt.density_gradient(P, v[:N], rhos, Ks, mu_ref)
    y = G.get("Y")
    for s in range(1, N):
        ref = w[s] - dens[s] / P.K
        assert rel(y[s], ref) < (1e-11 if prec == 1 else 2e-5), (s, rel(y[s], ref))


# ---------------------------------------------------------------------------
# a4: NSO residual f on every level
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("prec", PREC)
@pytest.mark.parametrize("shape,N", [((8, 8, 8), 3), ((12, 8, 8), 2), ((32, 32, 32), 2), ((40, 32, 24), 2)])
def test_nso_residual_3d_all_levels(prec, shape, N):
    """Levels of at least 50000 faces (32^3, 40 x 32 x 24) take the two-pass
    form (the Lamb-vector products stored per face, then gathered)."""
    nx, ny, nz = shape
    P, G = make_pair3(nx, ny, nz, N, precision=prec)
    grids = stfas.hierarchy(P)
    assert G.num_levels() == len(grids) >= 2
    for l, g in enumerate(grids):
        x = random_state3(P, 10 + l, grid=g)
        z = np.random.default_rng(20 + l).standard_normal((N, g.F)) * g.interior_faces()
        G.set_state(x, level=l)
        G.set("Z", z, level=l)
        inf = G.nso_residual(level=l)
        f = kkt.nso_residual(P, g, x, z)
        got = G.get_state(level=l, prefix="RES_")
        dbl = prec == 1 or (l == len(grids) - 1 and l > 0)
        for k in f:
            assert rel(got[k], f[k]) < (1e-12 if dbl else 2e-6), (l, k, rel(got[k], f[k]))
        assert abs(inf - kkt.state_inf(f)) <= (1e-12 if dbl else 1e-5) * kkt.state_inf(f)


# ---------------------------------------------------------------------------
# a8: SCGS sweep (8 colours, 7x7 blocks) with the temporal block-tridiagonal solve
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("prec", PREC)
@pytest.mark.parametrize("shape,N", [((8, 8, 8), 3), ((12, 8, 8), 5), ((6, 4, 4), 1)])
def test_scgs_sweep_3d(prec, shape, N):
    nx, ny, nz = shape
    P, G = make_pair3(nx, ny, nz, N, precision=prec, dt=1.0 / max(N, 16))
    grids = stfas.hierarchy(P)
    for l, g in enumerate(grids):
        x = random_state3(P, 30 + l, grid=g, scale=0.3)
        x["u"] *= 0.3
        z = np.random.default_rng(40 + l).standard_normal((N, g.F)) * g.interior_faces() * 0.3
        res = random_state3(P, 50 + l, grid=g, scale=0.1) if l > 0 else kkt.zero_state(P, g)
        if l > 0:
            res["v"][0] = 0.0
            res["pbar"][0] = 0.0
        G.set_state(x, level=l)
        G.set("Z", z, level=l)
        for k, name in (("v", "RES_IN_V"), ("pbar", "RES_IN_PBAR"), ("u", "RES_IN_U"), ("p", "RES_IN_P")):
            G.set(name, res[k], level=l)
        G.smooth(level=l, sweeps=1)
        got = G.get_state(level=l)
        ref = kkt.copy_state(x)
        scgs.sweep(P, g, ref, z, res)
        dbl = prec == 1
        for k in ref:
            d = ref[k] - x[k]
            err = np.linalg.norm(got[k] - ref[k])
            tol = TOL[1]["smooth"] if dbl else TOL[0]["smooth"]
            floor = 0.0 if dbl else 2e-7 * np.linalg.norm(x[k])
            assert err <= tol * np.linalg.norm(d) + floor, (l, k, err / max(np.linalg.norm(d), 1e-300))


@pytest.mark.parametrize("periodic", [False, True])
@pytest.mark.parametrize("prec", PREC)
def test_scgs_sweep_3d_thread_per_cell(prec, periodic):
    """A colour of >= 16384 cells runs the thread-per-cell block Thomas kernel
    (64 x 64 x 32: 16384 cells per colour on the finest level).  From the zero
    state towards a smooth target: the first sweep builds a velocity, the
    second runs with the Adv coupling of that velocity.  (A random state with
    O(1) pressures at h = 1/64 is amplified ~1e16-fold by the colour sweeps --
    no test of anything.)"""
    nx, ny, nz, N = 64, 64, 32, 2
    P, G = make_pair3(nx, ny, nz, N, precision=prec, periodic=periodic)
    z = velocity3(nx, ny, nz, N, amp=0.5, seed=45, periodic=periodic)[1:]
    G.set("Z", z)
    x = kkt.zero_state(P)
    res = kkt.zero_state(P, P.grid)
    for s in range(2):
        G.smooth(level=0, sweeps=1)
        scgs.sweep(P, P.grid, x, z, res)
        got = G.get_state()
        for k in x:
            assert rel(got[k], x[k]) < (1e-9 if prec == 1 else 2e-4), (s, k, rel(got[k], x[k]))


# ---------------------------------------------------------------------------
# a9: restriction and prolongation-correction
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("prec", PREC)
def test_transfers_3d(prec):
    nx, ny, nz, N = 12, 8, 8, 2
    P, G = make_pair3(nx, ny, nz, N, precision=prec)
    grids = stfas.hierarchy(P)
    x0 = random_state3(P, 60)
    G.set_state(x0, 0)
    G.restrict(0)
    xc = stfas.restrict_state(grids[0], x0)
    got = G.get_state(1)
    old = G.get_state(1, prefix="XOLD_")
    tol = 1e-14 if prec == 1 else 1e-6
    for k in xc:
        assert rel(got[k], xc[k]) < tol and rel(old[k], xc[k]) < tol, k
    xn = random_state3(P, 61, grid=grids[1])
    G.set_state(xn, 1)
    G.prolong_correct(0)
    corr = stfas.prolong_state(grids[0], grids[1], kkt.state_sub(xn, xc))
    corr["v"][0] = 0.0
    corr["pbar"][0] = 0.0
    got = G.get_state(0)
    for k in x0:
        assert rel(got[k], x0[k] + corr[k]) < tol * 10, k


# ---------------------------------------------------------------------------
# a10: full V-cycle (Alg. 2) from the AO target
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("prec", PREC)
@pytest.mark.parametrize("shape,N", [((8, 8, 8), 4), ((16, 8, 8), 3)])
def test_vcycle_3d(prec, shape, N):
    nx, ny, nz = shape
    P, G = make_pair3(nx, ny, nz, N, precision=prec, r=1e-3)
    v = velocity3(nx, ny, nz, N, amp=0.5, seed=5)
    lam = workloads.random_faces3(np.random.default_rng(6), nx, ny, nz, N, 0.05)
    lam[0] = 0.0
    G.set("VSTAR", v[:N])
    G.set("LAMBDA", lam)
    G.prepare_targets()
    z = v[:N] - lam / P.K
    x = kkt.zero_state(P)
    for c in range(2):
        f_gpu = G.vcycle(1)
        f_ref = stfas.stfas_cycle(P, x, z)
        got = G.get_state(0)
        for k in x:
            assert rel(got[k], x[k]) < TOL[prec]["vcycle"], (c, k, rel(got[k], x[k]))
        assert abs(f_gpu - f_ref) <= 1e-3 * f_ref + TOL[prec]["vcycle"] * 1e3


# ---------------------------------------------------------------------------
# KKT metric and a few ADMM iterations (Alg. 3) end to end
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("prec", PREC)
def test_kkt_residual_3d(prec):
    nx, ny, nz, N = 8, 8, 6, 4
    P, G = make_pair3(nx, ny, nz, N, precision=prec, levels=1, coarsest_n=2)
    v = velocity3(nx, ny, nz, N, amp=0.4, seed=9)
    v = np.array([projection.project(P.grid, a) for a in v])
    G.set("V", v)
    norm = G.kkt_residual()
    g_ref = kkt.reduced_gradient(P, v)
    u_ref = kkt.forces(P, v)
    tol = 2e-7 if prec == 1 else 2e-4
    assert rel(G.get("KKT_U"), u_ref) < tol
    g = G.get("KKT_G")
    assert rel(g[1:], g_ref[1:]) < tol, rel(g[1:], g_ref[1:])
    assert abs(norm - np.linalg.norm(g_ref)) <= tol * np.linalg.norm(g_ref)


@pytest.mark.parametrize("prec", PREC)
def test_ao_3d(prec):
    nx, ny, nz, N = 8, 8, 8, 4
    P, G = make_pair3(nx, ny, nz, N, precision=prec, levels=1, K=2.0)
    v = velocity3(nx, ny, nz, N, amp=0.4, seed=7)
    lam = workloads.random_faces3(np.random.default_rng(8), nx, ny, nz, N, 0.05)
    lam[0] = 0.0
    G.set("V", v)
    G.set("LAMBDA", lam)
    G.ao(2)
    trace_ref = []
    vs_ref, rhos_ref, _ = admm.ao(P, v, lam, iters=2, trace=trace_ref)
    assert G.ao_trace() == trace_ref, (G.ao_trace(), trace_ref)
    vs = G.get("VSTAR")
    for s in range(N):
        assert rel(vs[s], vs_ref[s]) < TOL[prec]["ao"] * 5, (s, rel(vs[s], vs_ref[s]))
    rho = G.get("RHO")
    for s in range(N + 1):
        assert rel(rho[s], rhos_ref[s]) < TOL[prec]["ao"] * 5


@pytest.mark.parametrize("prec", PREC)
def test_admm_iterations_3d(prec):
    nx, ny, nz, N = 8, 8, 8, 4
    P, G = make_pair3(nx, ny, nz, N, precision=prec, levels=1, r=1e-3)
    rep = G.solve(tol=1e-12, max_admm=2)
    x, vs, lam, hist = admm.solve(P, tol=1e-12, max_admm=2, eps_admm=P.rho_scale / 100)
    assert rep["admm_iters"] == len(hist)
    tol = 1e-5 if prec == 1 else 2e-3
    assert abs(rep["kkt_rel"] - hist[-1]["kkt_rel"]) <= tol * hist[-1]["kkt_rel"]
    v = G.get("V")
    assert rel(v, x["v"]) < tol, rel(v, x["v"])
    J_gpu = kkt.objective(P, v)
    J_ref = kkt.objective(P, x["v"])
    assert abs(J_gpu - J_ref) <= (1e-8 if prec == 1 else 1e-4) * J_ref
    # v is solenoidal up to the NSO residual (row 2 of f), as the oracle's iterate
    div_gpu = max(np.max(np.abs(mac.div(P.grid, a))) for a in v)
    div_ref = max(np.max(np.abs(mac.div(P.grid, a))) for a in x["v"])
    assert div_gpu <= 2 * div_ref + (1e-10 if prec == 1 else 1e-4), (div_gpu, div_ref)


# ---------------------------------------------------------------------------
# periodic boundaries (every axis wraps), the same steps against the oracle
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("prec", PREC)
def test_periodic_residual_transfers_and_sweep(prec):
    nx, ny, nz, N = 8, 8, 8, 3
    P, G = make_pair3(nx, ny, nz, N, precision=prec, periodic=True, dt=1.0 / 16)
    grids = stfas.hierarchy(P)
    for l, g in enumerate(grids):
        x = random_state3(P, 110 + l, grid=g, scale=0.3)
        x["u"] *= 0.3
        z = np.random.default_rng(120 + l).standard_normal((N, g.F)) * g.interior_faces() * 0.3
        G.set_state(x, level=l)
        G.set("Z", z, level=l)
        G.nso_residual(level=l)
        f = kkt.nso_residual(P, g, x, z)
        got = G.get_state(level=l, prefix="RES_")
        dbl = prec == 1 or (l == len(grids) - 1 and l > 0)
        for k in f:
            assert rel(got[k], f[k]) < (1e-12 if dbl else 2e-6), (l, k, rel(got[k], f[k]))
        res = kkt.zero_state(P, g)
        G.smooth(level=l, sweeps=1)
        ref = kkt.copy_state(x)
        scgs.sweep(P, g, ref, z, res)
        got = G.get_state(level=l)
        for k in ref:
            d = ref[k] - x[k]
            err = np.linalg.norm(got[k] - ref[k])
            tol = TOL[1]["smooth"] if prec == 1 else TOL[0]["smooth"]
            floor = 0.0 if prec == 1 else 2e-7 * np.linalg.norm(x[k])
            assert err <= tol * np.linalg.norm(d) + floor, (l, k, err / max(np.linalg.norm(d), 1e-300))
    x0 = random_state3(P, 130)
    G.set_state(x0, 0)
    G.restrict(0)
    xc = stfas.restrict_state(grids[0], x0)
    got = G.get_state(1)
    tol = 1e-14 if prec == 1 else 1e-6
    for k in xc:
        assert rel(got[k], xc[k]) < tol, k
    xn = random_state3(P, 131, grid=grids[1])
    G.set_state(xn, 1)
    G.prolong_correct(0)
    corr = stfas.prolong_state(grids[0], grids[1], kkt.state_sub(xn, xc))
    corr["v"][0] = 0.0
    corr["pbar"][0] = 0.0
    got = G.get_state(0)
    for k in x0:
        assert rel(got[k], x0[k] + corr[k]) < tol * 10, k


@pytest.mark.parametrize("prec", PREC)
def test_periodic_advection_adjoint_and_projection(prec):
    nx, ny, nz, N = 8, 8, 8, 4
    mid = workloads.gaussian_ball3(nx, ny, nz, (0.1, 0.5, 0.5), 0.12)     # straddles the wrap
    end = workloads.gaussian_ball3(nx, ny, nz, (0.9, 0.6, 0.4), 0.12)
    kf = {N // 2: (mid, 0.5), N: (end, 1.0)}
    P, G = make_pair3(nx, ny, nz, N, precision=prec, levels=2, keyframes=kf, K=2.0, periodic=True)
    rng = np.random.default_rng(140)
    v = np.zeros((N + 1, P.grid.F))
    v[1:] = rng.standard_normal((N, P.grid.F)) * P.grid.interior_faces() * 0.4
    v[:, :P.grid.Fx] += 0.6 * P.grid.interior_faces()[:P.grid.Fx]   # a mean flow across the wrap
    w = rng.standard_normal((N, P.grid.F)) * P.grid.interior_faces() * 0.2
    G.set("VSTAR", v[:N])
    G.set("W", w)
    G.advect("VSTAR")
    G.metric_terms()
    G.adjoint("VSTAR", 1.0, 1.0 / P.K)
    rhos, Ks = kkt.forward_density(P, v[:N])
    np.testing.assert_array_equal(G.taylor_orders(), Ks)
    rho = G.get("RHO")
    for i in range(N + 1):
        assert rel(rho[i], rhos[i]) < (1e-12 if prec == 1 else 1e-5), i
    mt = G.get("MTERM")
    for s in kf:
        assert rel(mt[s], P.misfit_grad(s, rhos[s])) < (1e-11 if prec == 1 else 2e-5), s
    mu_ref = kkt.adjoint_density(P, v[:N], rhos, Ks)
    mu = G.get("MU")
    for s in range(N):
        assert rel(mu[s], mu_ref[s]) < (1e-11 if prec == 1 else 2e-5), s
    dens = kkt.density_gradient(P, v[:N], rhos, Ks, mu_ref)
    y = G.get("Y")
    for s in range(1, N):
        assert rel(y[s], w[s] - dens[s] / P.K) < (1e-11 if prec == 1 else 2e-5), s
    # projection of 3 fields (the constant x-flow is harmonic and survives)
    G.set("W", w)
    G.project("W", 0, 3)
    out = G.get("W")
    for i in range(3):
        ref = projection.project(P.grid, w[i])
        assert rel(out[i], ref) < TOL[prec]["project"] * 5, (i, rel(out[i], ref))


@pytest.mark.parametrize("prec", PREC)
def test_periodic_vcycle_kkt_and_admm(prec):
    nx, ny, nz, N = 8, 8, 8, 4
    P, G = make_pair3(nx, ny, nz, N, precision=prec, r=1e-3, periodic=True)
    v = velocity3(nx, ny, nz, N, amp=0.5, seed=150, periodic=True)
    lam = workloads.random_faces3(np.random.default_rng(151), nx, ny, nz, N, 0.05, periodic=True)
    lam[0] = 0.0
    G.set("VSTAR", v[:N])
    G.set("LAMBDA", lam)
    G.prepare_targets()
    z = v[:N] - lam / P.K
    x = kkt.zero_state(P)
    for c in range(2):
        f_gpu = G.vcycle(1)
        f_ref = stfas.stfas_cycle(P, x, z)
        got = G.get_state(0)
        for k in x:
            assert rel(got[k], x[k]) < TOL[prec]["vcycle"], (c, k, rel(got[k], x[k]))
        assert abs(f_gpu - f_ref) <= 1e-3 * f_ref + TOL[prec]["vcycle"] * 1e3
    vs = np.array([projection.project(P.grid, a) for a in v])
    G.set("V", vs)
    norm = G.kkt_residual()
    g_ref = kkt.reduced_gradient(P, vs)
    tol = 2e-7 if prec == 1 else 2e-4
    assert rel(G.get("KKT_G")[1:], g_ref[1:]) < tol
    assert abs(norm - np.linalg.norm(g_ref)) <= tol * np.linalg.norm(g_ref)
    P2, G2 = make_pair3(nx, ny, nz, N, precision=prec, r=1e-3, periodic=True)
    rep = G2.solve(tol=1e-12, max_admm=2)
    xs, _, _, hist = admm.solve(P2, tol=1e-12, max_admm=2, eps_admm=P2.rho_scale / 100)
    tol = 1e-5 if prec == 1 else 2e-3
    assert rep["admm_iters"] == len(hist)
    assert abs(rep["kkt_rel"] - hist[-1]["kkt_rel"]) <= tol * hist[-1]["kkt_rel"]
    assert rel(G2.get("V"), xs["v"]) < tol


def test_periodic_parameters_are_validated():
    with pytest.raises(stc.StcError):
        make_pair3(8, 8, 6 + 1, 2, periodic=True)          # odd nz breaks the parity colours
    prm = stc.default_params(16, 16, 4, boundary=1)       # 2D: periodic is a 3D option
    with pytest.raises(stc.StcError):
        stc.Problem(prm, np.ones(256))
