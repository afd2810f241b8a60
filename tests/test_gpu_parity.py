"""GPU parity: every step of the hot path, called through the C ABI of libstc,
against the fp64 oracle on the same seeded inputs.

fp64 mode (precision=1) must agree to rounding (plus the projection's multigrid
truncation); fp32 mode (precision=0) within the precision policy's bounds (see
gpu_common.TOL).  Grids span several colour tiles and ragged shapes.
"""
import numpy as np
import pytest

from oracle import admm, kkt, mac, projection, scgs, stfas
from paper_1608_01102_gb300 import stc, workloads

from gpu_common import TOL, make_pair, random_state, rel, velocity_trajectory

pytestmark = [pytest.mark.gpu, pytest.mark.filterwarnings("ignore::DeprecationWarning")]

PREC = [1, 0]


# ---------------------------------------------------------------------------
# a2: projection Q
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("prec", PREC)
@pytest.mark.parametrize("shape", [(16, 16), (24, 12), (32, 32)])
def test_projection(prec, shape):
    nx, ny = shape
    P, G = make_pair(nx, ny, N=4, precision=prec)
    rng = np.random.default_rng(1)
    w = workloads.random_faces(rng, nx, ny, 4)
    w[1] += workloads.swirl_velocity(nx, ny, 3.0)
    G.set("W", w)
    G.project("W", 0, 4)
    out = G.get("W")
    for i in range(4):
        ref = projection.project(P.grid, w[i])
        assert rel(out[i], ref) < TOL[prec]["project"], (i, rel(out[i], ref))
        d = mac.div(P.grid, out[i])
        assert np.max(np.abs(d)) < TOL[prec]["project"] * np.max(np.abs(mac.div(P.grid, w[i]))) * 10


@pytest.mark.parametrize("prec", PREC)
@pytest.mark.parametrize("shape", [(16, 16), (24, 12), (10, 6), (48, 48), (128, 96)])
def test_projection_is_exact_where_the_dct_applies(prec, shape):
    """2D fields that fit on chip are projected through the DCT-II
    diagonalisation of the Neumann Laplacian: Q itself to rounding, against the
    oracle's sparse direct solve (10 x 6: the scalar path of the products;
    128 x 96: a non-square bench-sized grid).  Q is idempotent and leaves
    divergence at the rounding level."""
    nx, ny = shape
    P, G = make_pair(nx, ny, N=3, precision=prec, levels=0)
    rng = np.random.default_rng(3)
    w = workloads.random_faces(rng, nx, ny, 3)
    w[1] += workloads.swirl_velocity(nx, ny, 3.0)
    G.set("W", w)
    G.project("W", 0, 3)
    out = G.get("W")
    tol = 1e-12 if prec == 1 else 5e-6
    for i in range(3):
        ref = projection.project(P.grid, w[i])
        assert rel(out[i], ref) < tol, (i, rel(out[i], ref))
        assert np.max(np.abs(mac.div(P.grid, out[i]))) < tol * np.max(np.abs(mac.div(P.grid, w[i]))) * 100
    G.set("W", out)
    G.project("W", 0, 3)
    again = G.get("W")
    for i in range(3):
        assert rel(again[i], out[i]) < tol, i


def test_problem_created_on_a_busy_stream_projects_exactly():
    """Everything a problem uploads at creation is ordered after the zeroing
    of its buffers on the problem's own stream: created on a non-blocking
    stream that is still busy, the projection tables must hold (a copy issued
    on another stream would land before the queued memset and be erased)."""
    torch = pytest.importorskip("torch")
    nx = ny = 32
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        torch.cuda._sleep(200_000_000)            # ~0.1 s of GPU time ahead of the problem's setup
    P, _ = make_pair(nx, ny, N=2, precision=1, levels=0)
    prm = stc.default_params(nx, ny, 2, precision=1, r=1e-2, K=1.0, metric_levels=0)
    G = stc.Problem(prm, P.rho0, stream=s.cuda_stream)
    w = workloads.random_faces(np.random.default_rng(5), nx, ny, 2)
    w[1] += workloads.swirl_velocity(nx, ny, 3.0)
    G.set("W", w)
    G.project("W", 0, 2)
    out = G.get("W")
    for i in range(2):
        assert rel(out[i], projection.project(P.grid, w[i])) < 1e-12, i
    G.close()


def test_projection_with_global_scratch_fp64_128():
    """128^2 in fp64 does not fit the on-chip multigrid layout: the level
    arrays move to a per-field global scratch (same arithmetic)."""
    nx = ny = 128
    P, G = make_pair(nx, ny, N=2, precision=1, levels=0)
    rng = np.random.default_rng(2)
    w = workloads.random_faces(rng, nx, ny, 2)
    w[1] += workloads.swirl_velocity(nx, ny, 3.0)
    G.set("W", w)
    G.project("W", 0, 2)
    out = G.get("W")
    for i in range(2):
        ref = projection.project(P.grid, w[i])
        assert rel(out[i], ref) < TOL[1]["project"] * 10, (i, rel(out[i], ref))


# ---------------------------------------------------------------------------
# a3: forward advection (Taylor exponential, adaptive order)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("prec", PREC)
@pytest.mark.parametrize("shape,N", [((16, 16), 6), ((24, 12), 5), ((32, 32), 8), ((32, 24), 4), ((12, 8), 3)])
def test_forward_advection(prec, shape, N):
    nx, ny = shape
    P, G = make_pair(nx, ny, N=N, precision=prec)
    v = velocity_trajectory(nx, ny, N, amp=0.8)
    G.set("VSTAR", v[:N])
    G.advect("VSTAR")
    rho = G.get("RHO")
    K = G.taylor_orders()
    ref, Kref = kkt.forward_density(P, v[:N])
    np.testing.assert_array_equal(K, Kref)
    assert max(Kref) > 3
    for i in range(N + 1):
        assert rel(rho[i], ref[i]) < (1e-12 if prec == 1 else 1e-5), (i, rel(rho[i], ref[i]))
    # mass is conserved exactly up to rounding
    assert abs(rho[N].sum() - P.rho0.sum()) < (1e-10 if prec == 1 else 1e-4) * P.rho0.sum()


# ---------------------------------------------------------------------------
# a5 / a6 / a7: keyframe metric, backward adjoint sweep, v*-gradient
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("prec", PREC)
@pytest.mark.parametrize("shape,N,levels", [((16, 16), 6, 2), ((24, 12), 5, 1), ((32, 32), 6, 3),
                                            ((32, 24), 4, 2), ((12, 8), 3, 1), ((16, 12), 3, 5)])
def test_adjoint_sweep(prec, shape, N, levels):
    nx, ny = shape
    star_mid = workloads.gaussian_ball(nx, ny, (0.4, 0.5 * ny / nx), 0.1)
    star_end = workloads.gaussian_ball(nx, ny, (0.6, 0.6 * ny / nx), 0.1)
    kf = {N // 2: (star_mid, 0.5), N: (star_end, 1.0)}
    P, G = make_pair(nx, ny, N=N, precision=prec, levels=levels, keyframes=kf, K=2.0)
    v = velocity_trajectory(nx, ny, N, amp=0.7, seed=3)
    rng = np.random.default_rng(4)
    w = workloads.random_faces(rng, nx, ny, N, 0.2)
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
            assert rel(mt[s], ref) < (1e-11 if prec == 1 else 2e-5)
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
@pytest.mark.parametrize("shape,N", [((16, 16), 4), ((24, 16), 3)])
def test_nso_residual_all_levels(prec, shape, N):
    nx, ny = shape
    P, G = make_pair(nx, ny, N=N, precision=prec)
    grids = stfas.hierarchy(P)
    assert G.num_levels() == len(grids)
    for l, g in enumerate(grids):
        x = random_state(P, 10 + l, grid=g)
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
# a8: SCGS sweep (all colours) with the temporal block-tridiagonal solve
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("prec", PREC)
@pytest.mark.parametrize("shape,N", [((16, 16), 5), ((12, 8), 3), ((8, 8), 1)])
def test_scgs_sweep(prec, shape, N):
    nx, ny = shape
    # a physical timestep (dt = 1 with a random state makes one Gauss-Seidel
    # sweep amplify the state 1e4-fold, a test artefact rather than a case)
    P, G = make_pair(nx, ny, N=N, precision=prec, dt=1.0 / max(N, 16))
    grids = stfas.hierarchy(P)
    for l, g in enumerate(grids):
        x = random_state(P, 30 + l, grid=g, scale=0.3)
        x["u"] *= 0.3
        z = np.random.default_rng(40 + l).standard_normal((N, g.F)) * g.interior_faces() * 0.3
        res = random_state(P, 50 + l, grid=g, scale=0.1) if l > 0 else kkt.zero_state(P, g)
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
        dbl = prec == 1   # the fp32 mode solves even the fp64 coarsest level's corrections in fp32
        for k in ref:
            # compare the update itself; in fp32 the stored state carries its own
            # rounding (eps * |x|), which bounds how well a small update can agree
            d = ref[k] - x[k]
            err = np.linalg.norm(got[k] - ref[k])
            tol = TOL[1]["smooth"] if dbl else TOL[0]["smooth"]
            floor = 0.0 if dbl else 2e-7 * np.linalg.norm(x[k])
            assert err <= tol * np.linalg.norm(d) + floor, (l, k, err / max(np.linalg.norm(d), 1e-300))


@pytest.mark.parametrize("prec", PREC)
def test_warp_and_cta_per_cell_smoothers_agree(prec):
    """The two 2D smoother kernels solve the same local systems: one warp per
    cell (the nine-column saddle solve per lane) and one CTA per cell (the
    block steps split over its threads, one column per thread).  Per level
    and through whole V-cycles on 32^2 x 8 they agree to rounding (the split
    repeats the same arithmetic per column, so in practice bit for bit)."""
    nx, ny, N = 32, 32, 8
    v = velocity_trajectory(nx, ny, N, amp=0.5, seed=61)
    lam = workloads.random_faces(np.random.default_rng(62), nx, ny, N, 0.05)
    lam[0] = 0.0
    out = {}
    for name, over in (("cta", dict()), ("warp", dict(scgs_cta_cells=0))):
        P, G = make_pair(nx, ny, N=N, precision=prec, dt=1.0 / 16, **over)
        G.set("VSTAR", v[:N])
        G.set("LAMBDA", lam)
        G.prepare_targets()
        states = []
        for l in range(G.num_levels()):
            g = stfas.hierarchy(P)[l]
            G.set_state(random_state(P, 70 + l, grid=g, scale=0.3), level=l)
            G.smooth(level=l, sweeps=2)
            states.append(G.get_state(level=l))
        G.set_state(kkt.zero_state(P))
        f = [G.vcycle(1) for _ in range(3)]
        out[name] = (states, f, G.get_state())
        G.close()
    (sa, fa, xa), (sb, fb, xb) = out["cta"], out["warp"]
    for l, (a, b) in enumerate(zip(sa, sb)):
        for k in a:
            assert rel(a[k], b[k]) <= TOL[prec]["smooth"], (l, k, rel(a[k], b[k]))
    for a, b in zip(fa, fb):
        assert abs(a - b) <= TOL[prec]["vcycle"] * abs(b), (fa, fb)
    for k in xa:
        assert rel(xa[k], xb[k]) <= TOL[prec]["vcycle"], (k, rel(xa[k], xb[k]))


# ---------------------------------------------------------------------------
# a9: restriction and prolongation-correction
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("prec", PREC)
def test_transfers(prec):
    nx, ny, N = 16, 12, 3
    P, G = make_pair(nx, ny, N=N, precision=prec)
    grids = stfas.hierarchy(P)
    x0 = random_state(P, 60)
    G.set_state(x0, 0)
    G.restrict(0)
    xc = stfas.restrict_state(grids[0], x0)
    got = G.get_state(1)
    old = G.get_state(1, prefix="XOLD_")
    tol = 1e-14 if prec == 1 else 1e-6
    for k in xc:
        assert rel(got[k], xc[k]) < tol and rel(old[k], xc[k]) < tol
    xn = random_state(P, 61, grid=grids[1])
    G.set_state(xn, 1)
    G.prolong_correct(0)
    corr = stfas.prolong_state(grids[0], grids[1], kkt.state_sub(xn, xc))
    corr["v"][0] = 0.0
    corr["pbar"][0] = 0.0
    got = G.get_state(0)
    for k in x0:
        assert rel(got[k], x0[k] + corr[k]) < tol, k


# ---------------------------------------------------------------------------
# a14: time coarsening (opt-in): hierarchy, transfers in space and time, V-cycle
# ---------------------------------------------------------------------------
def _tc_random_state(P, seed, g, N):
    rng = np.random.default_rng(seed)
    m = g.interior_faces()
    x = dict(v=rng.standard_normal((N + 1, g.F)) * m, pbar=rng.standard_normal((N + 1, g.C)),
             u=rng.standard_normal((N, g.F)) * m, p=rng.standard_normal((N, g.C)))
    x["v"][0] = 0.0
    x["pbar"][0] = 0.0
    return x


@pytest.mark.parametrize("prec", PREC)
def test_time_coarsened_hierarchy_and_transfers(prec):
    nx, ny, N = 16, 12, 8
    P, G = make_pair(nx, ny, N=N, precision=prec, time_coarsen=True)
    lv = stfas.levels(P)
    assert G.num_levels() == len(lv)
    for l, (g, Pl) in enumerate(lv):
        n, dt = G.level_steps(l)
        assert n == Pl.N and dt == pytest.approx(Pl.dt, rel=1e-15)
    (g0, P0), (g1, P1) = lv[0], lv[1]
    assert P1.N == N // 2
    x0 = _tc_random_state(P, 62, g0, N)
    G.set_state(x0, 0)
    G.restrict(0)
    xc = stfas.restrict_state_st(g0, x0, True)
    got = G.get_state(1)
    tol = 1e-14 if prec == 1 else 1e-6
    for k in xc:
        assert got[k].shape == xc[k].shape and rel(got[k], xc[k]) < tol, k
    xn = _tc_random_state(P, 63, g1, P1.N)
    G.set_state(xn, 1)
    G.prolong_correct(0)
    corr = stfas.prolong_state_st(g0, g1, kkt.state_sub(xn, xc), True)
    corr["v"][0] = 0.0
    corr["pbar"][0] = 0.0
    got = G.get_state(0)
    for k in x0:
        assert rel(got[k], x0[k] + corr[k]) < tol * 10, k
    # the targets restrict as point fields without an end point
    z = workloads.random_faces(np.random.default_rng(64), nx, ny, N)
    G.set("VSTAR", z)
    G.set("LAMBDA", np.zeros_like(z))
    G.prepare_targets()
    zc = stfas.restrict_targets(g0, z, True)
    assert rel(G.get("Z", 1), zc) < tol


@pytest.mark.parametrize("prec", PREC)
def test_time_coarsened_vcycle(prec):
    nx, ny, N = 16, 16, 8
    P, G = make_pair(nx, ny, N=N, precision=prec, r=1e-3, time_coarsen=True)
    assert [G.level_steps(l)[0] for l in range(G.num_levels())] == [Pl.N for _, Pl in stfas.levels(P)]
    v = velocity_trajectory(nx, ny, N, amp=0.5, seed=5)
    lam = workloads.random_faces(np.random.default_rng(6), nx, ny, N, 0.05)
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
# a10: full V-cycle (Alg. 2) from the AO target
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("prec", PREC)
@pytest.mark.parametrize("shape,N", [((16, 16), 6), ((32, 32), 8), ((24, 16), 4)])
def test_vcycle(prec, shape, N):
    nx, ny = shape
    P, G = make_pair(nx, ny, N=N, precision=prec, r=1e-3)
    v = velocity_trajectory(nx, ny, N, amp=0.5, seed=5)
    lam = workloads.random_faces(np.random.default_rng(6), nx, ny, N, 0.05)
    lam[0] = 0.0
    G.set("VSTAR", v[:N])
    G.set("LAMBDA", lam)
    G.prepare_targets()
    z = v[:N] - lam / P.K
    np.testing.assert_allclose(G.get("Z"), z, rtol=1e-6 if prec == 0 else 1e-14, atol=1e-7)
    x = kkt.zero_state(P)
    for c in range(2):
        f_gpu = G.vcycle(1)
        f_ref = stfas.stfas_cycle(P, x, z)
        got = G.get_state(0)
        for k in x:
            assert rel(got[k], x[k]) < TOL[prec]["vcycle"], (c, k, rel(got[k], x[k]))
        assert abs(f_gpu - f_ref) <= 1e-3 * f_ref + TOL[prec]["vcycle"] * 1e3


@pytest.mark.parametrize("prec", PREC)
def test_vcycle_plain_alg2(prec):
    """Alg. 2 exactly as printed: no coarse-correction guard, no damping
    (omega = 1) and the Eq. HESS local blocks without a Levenberg-Marquardt
    shift (lm_shift = 0, no adaptation) -- none of the safeguards that the
    library and the oracle turn on by default.  Three cycles from zero."""
    nx, ny, N = 16, 16, 6
    P, G = make_pair(nx, ny, N=N, precision=prec, r=1e-3, cgc_guard=False, scgs_omega=1.0, lm_shift=0.0,
                     lm_adapt=False)
    assert P.lm_shift == 0.0 and P.omega == 1.0 and not P.cgc_guard
    v = velocity_trajectory(nx, ny, N, amp=1.0, seed=5)
    lam = workloads.random_faces(np.random.default_rng(6), nx, ny, N, 0.05)
    lam[0] = 0.0
    G.set("VSTAR", v[:N])
    G.set("LAMBDA", lam)
    G.prepare_targets()
    z = v[:N] - lam / P.K
    x = kkt.zero_state(P)
    f_prev = np.inf
    for c in range(3):
        f_gpu = G.vcycle(1)
        f_ref = stfas.stfas_cycle(P, x, z)
        assert f_ref < 0.2 * f_prev       # the plain cycle contracts on this problem
        f_prev = f_ref
        got = G.get_state(0)
        for k in x:
            assert rel(got[k], x[k]) < TOL[prec]["vcycle"], (c, k, rel(got[k], x[k]))
        assert abs(f_gpu - f_ref) <= 1e-3 * f_ref + TOL[prec]["vcycle"] * 1e3


# ---------------------------------------------------------------------------
# Alg. 1: AO fixed point (forward, adjoint, projection) and targets
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("prec", PREC)
def test_ao(prec):
    nx, ny, N = 16, 16, 6
    P, G = make_pair(nx, ny, N=N, precision=prec, levels=2, K=2.0)
    v = velocity_trajectory(nx, ny, N, amp=0.4, seed=7)
    lam = workloads.random_faces(np.random.default_rng(8), nx, ny, N, 0.05)
    lam[0] = 0.0
    G.set("V", v)
    G.set("LAMBDA", lam)
    G.ao(2)
    trace_ref = []
    vs_ref, rhos_ref, _ = admm.ao(P, v, lam, iters=2, trace=trace_ref)
    # the blend decisions (halvings per pass) are integers: identical
    assert G.ao_trace() == trace_ref, (G.ao_trace(), trace_ref)
    vs = G.get("VSTAR")
    for s in range(N):
        assert rel(vs[s], vs_ref[s]) < TOL[prec]["ao"], (s, rel(vs[s], vs_ref[s]))
    rho = G.get("RHO")
    for s in range(N + 1):
        assert rel(rho[s], rhos_ref[s]) < TOL[prec]["ao"]
    z = G.get("Z")
    assert rel(z, vs_ref - lam / P.K) < TOL[prec]["ao"]
    # warm start: continue the fixed-point iteration from the current v*
    G.ao(2, warm=True)
    trace2 = []
    vs2_ref, _, _ = admm.ao(P, v, lam, iters=2, start=vs_ref, trace=trace2)
    assert G.ao_trace() == trace2
    vs2 = G.get("VSTAR")
    for s in range(N):
        assert rel(vs2[s], vs2_ref[s]) < 2 * TOL[prec]["ao"], (s, rel(vs2[s], vs2_ref[s]))


@pytest.mark.parametrize("prec", PREC)
def test_ao_blend_halvings(prec):
    """Sec. 5's blend with several halvings per pass (a small K makes the full
    fixed-point step overshoot; some trials exceed taylor_kmax and count as
    rejected).  The oracle's decisions have margins >= 3e-5 relative here, far
    above the fp32 rounding of the objective."""
    nx, ny, N = 16, 16, 6
    P, G = make_pair(nx, ny, N=N, precision=prec, levels=2, K=0.2)
    v = velocity_trajectory(nx, ny, N, amp=0.4, seed=7)
    lam = workloads.random_faces(np.random.default_rng(8), nx, ny, N, 0.05)
    lam[0] = 0.0
    G.set("V", v)
    G.set("LAMBDA", lam)
    G.ao(4)
    trace_ref = []
    vs_ref, rhos_ref, ks_ref = admm.ao(P, v, lam, iters=4, trace=trace_ref)
    assert max(trace_ref) >= 2
    assert G.ao_trace() == trace_ref, (G.ao_trace(), trace_ref)
    assert list(G.taylor_orders()) == list(ks_ref)
    vs = G.get("VSTAR")
    for s in range(N):
        assert rel(vs[s], vs_ref[s]) < TOL[prec]["ao"], (s, rel(vs[s], vs_ref[s]))
    rho = G.get("RHO")
    for s in range(N + 1):
        assert rel(rho[s], rhos_ref[s]) < TOL[prec]["ao"]


@pytest.mark.parametrize("trials", [1, 2, 3, 8])
def test_ao_blend_trials_at_once_match_one_at_a_time(trials):
    """The blend factors tried at once (in rounds of `trials`, each on its own
    stream and buffers) take the same factor as the oracle's one-at-a-time
    search, and the state is bit-identical to the library's own one-at-a-time
    search (stc_params.ao_trials = 1), rejected Taylor overflows included."""
    nx, ny, N = 16, 16, 6
    v = velocity_trajectory(nx, ny, N, amp=0.4, seed=7)
    lam = workloads.random_faces(np.random.default_rng(8), nx, ny, N, 0.05)
    lam[0] = 0.0
    out = {}
    for t in (1, trials):
        P, G = make_pair(nx, ny, N=N, precision=0, levels=2, K=0.2, ao_trials=t)
        G.set("V", v)
        G.set("LAMBDA", lam)
        G.ao(4)
        out[t] = (G.ao_trace(), G.get("VSTAR"), G.get("RHO"), G.get("MTERM"), list(G.taylor_orders()))
        G.close()
    trace_ref = []
    admm.ao(P, v, lam, iters=4, trace=trace_ref)
    assert max(trace_ref) >= 2
    assert out[trials][0] == out[1][0] == trace_ref
    for a, b in zip(out[trials][1:], out[1][1:]):
        np.testing.assert_array_equal(a, b)


@pytest.mark.parametrize("prec", PREC)
def test_ao_plain(prec):
    """ao_halvings = -1: the plain Alg. 1 (v* = y every pass)."""
    nx, ny, N = 16, 16, 6
    P, G = make_pair(nx, ny, N=N, precision=prec, levels=2, K=2.0, ao_halvings=-1)
    v = velocity_trajectory(nx, ny, N, amp=0.4, seed=7)
    lam = workloads.random_faces(np.random.default_rng(8), nx, ny, N, 0.05)
    lam[0] = 0.0
    G.set("V", v)
    G.set("LAMBDA", lam)
    G.ao(2)
    trace_ref = []
    vs_ref, rhos_ref, _ = admm.ao(P, v, lam, iters=2, trace=trace_ref)
    assert G.ao_trace() == trace_ref == [0, 0]
    vs = G.get("VSTAR")
    for s in range(N):
        assert rel(vs[s], vs_ref[s]) < TOL[prec]["ao"], (s, rel(vs[s], vs_ref[s]))
    rho = G.get("RHO")
    for s in range(N + 1):
        assert rel(rho[s], rhos_ref[s]) < TOL[prec]["ao"]


# ---------------------------------------------------------------------------
# KKT metric: reduced gradient g(v)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("prec", PREC)
def test_kkt_residual(prec):
    nx, ny, N = 16, 16, 5
    P, G = make_pair(nx, ny, N=N, precision=prec, levels=2, r=1e-2)
    v = velocity_trajectory(nx, ny, N, amp=0.4, seed=9)
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


# ---------------------------------------------------------------------------
# Alg. 3: a few ADMM iterations end to end
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("prec", PREC)
def test_admm_iterations(prec):
    nx, ny, N = 16, 16, 6
    P, G = make_pair(nx, ny, N=N, precision=prec, levels=2, r=1e-3, sigma=0.12)
    rep = G.solve(tol=1e-12, max_admm=3)
    x, vs, lam, hist = admm.solve(P, tol=1e-12, max_admm=3, eps_admm=P.rho_scale / 100)
    assert rep["admm_iters"] == len(hist)
    tol = 1e-5 if prec == 1 else 1e-3
    assert abs(rep["kkt_rel"] - hist[-1]["kkt_rel"]) <= tol * hist[-1]["kkt_rel"]
    v = G.get("V")
    assert rel(v, x["v"]) < tol, rel(v, x["v"])
    u = G.get("U")
    assert rel(u, x["u"]) < (tol if prec == 1 else 1e-3)
    J_gpu = kkt.objective(P, v)
    J_ref = kkt.objective(P, x["v"])
    assert abs(J_gpu - J_ref) <= (1e-8 if prec == 1 else 1e-4) * J_ref


@pytest.mark.parametrize("prec", PREC)
def test_admm_al_fallback(prec):
    """Sec. 5's AL fallback: the same multiplier-update decisions and the same
    iterate as the oracle (decisions with a clear margin on this case)."""
    nx, ny, N = 16, 16, 6
    P, G = make_pair(nx, ny, N=N, precision=prec, levels=2, r=1e-3, sigma=0.12, al_threshold=0.15)
    rep = G.solve(tol=1e-12, max_admm=5)
    x, vs, lam, hist = admm.solve(P, tol=1e-12, max_admm=5, eps_admm=P.rho_scale / 100)
    assert rep["admm_iters"] == len(hist)
    assert rep["lambda_updates"] == hist[-1]["lambda_updates"]
    tol = 1e-5 if prec == 1 else 1e-3
    assert abs(rep["objective"] - hist[-1]["objective"]) <= tol * hist[-1]["objective"]
    assert rel(G.get("V"), x["v"]) < tol
    assert rel(G.get("LAMBDA")[1:], lam[1:]) < (tol if prec == 1 else 1e-2) or np.all(lam == 0)


@pytest.mark.parametrize("prec", PREC)
def test_admm_adaptive_penalty(prec):
    """k_adapt: the same penalty decisions (K = 4, 4, 2, 1, 0.5, 0.25 on this
    case; every r_p / r_d ratio at least a factor 1.7 from the switching
    thresholds) and the same iterate as the oracle after 6 ADMM iterations."""
    nx, ny, N = 16, 16, 6
    P, G = make_pair(nx, ny, N=N, precision=prec, levels=2, r=1e-3, sigma=0.12, K=4.0, k_adapt=True)
    rep = G.solve(tol=1e-12, max_admm=6)
    x, vs, lam, hist = admm.solve(P, tol=1e-12, max_admm=6, eps_admm=P.rho_scale / 100)
    assert [h["K"] for h in hist] == [4.0, 4.0, 2.0, 1.0, 0.5, 0.25]
    assert rep["admm_iters"] == len(hist) and rep["K_final"] == hist[-1]["K"]
    tol = 1e-5 if prec == 1 else 1e-3
    assert abs(rep["kkt_rel"] - hist[-1]["kkt_rel"]) <= tol * hist[-1]["kkt_rel"]
    assert rel(G.get("V"), x["v"]) < tol
    assert rel(G.get("U"), x["u"]) < (tol if prec == 1 else 1e-3)


# ---------------------------------------------------------------------------
# Sec. 5 LM safeguard of the NSO loop on a rough target: the first cycle at the
# default shift blows up on both sides and is undone, the raised shift converges
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("prec", PREC)
def test_nso_solve_lm_safeguard(prec):
    nx, ny, N = 16, 16, 4
    P, G = make_pair(nx, ny, N=N, precision=prec, levels=2, r=1e-3, K=1.0)
    z = workloads.random_faces(np.random.default_rng(0), nx, ny, N, 1.0)
    z[0] = 0.0
    G.set("VSTAR", z)
    G.set("LAMBDA", np.zeros_like(z))
    G.prepare_targets()
    x = kkt.zero_state(P)
    lm = dict(gamma=P.lm_shift, gamma0=P.lm_shift, rejected=0)
    f_ref, c_ref = admm.nso(P, x, z, 1.0, 0.0, 6, lm)
    f_gpu, c_gpu = G.nso_solve(0.0, 6)
    gamma, rejected = G.lm_info()
    assert lm["rejected"] >= 1 and c_gpu == c_ref == 6
    assert rejected == lm["rejected"] and gamma == lm["gamma"], (rejected, gamma, lm)
    got = G.get_state()
    tol = 1e-8 if prec == 1 else 2e-3
    for k in x:
        assert rel(got[k], x[k]) < tol, (k, rel(got[k], x[k]))
    assert abs(f_gpu - f_ref) <= tol * f_ref * 10


# ---------------------------------------------------------------------------
# edge cases
# ---------------------------------------------------------------------------
def test_single_level_grid_and_single_step():
    P, G = make_pair(4, 4, N=1, precision=1)
    assert G.num_levels() == 1
    x = random_state(P, 70)
    z = np.random.default_rng(71).standard_normal((1, P.grid.F)) * P.grid.interior_faces()
    G.set_state(x)
    G.set("Z", z)
    G.smooth(0, 2)
    ref = kkt.copy_state(x)
    res = kkt.zero_state(P)
    for _ in range(2):
        scgs.sweep(P, P.grid, ref, z, res)
    got = G.get_state()
    for k in ref:
        assert rel(got[k], ref[k]) < 1e-10


def test_no_keyframes_gives_zero_adjoint():
    P, G = make_pair(16, 16, N=4, precision=0, keyframes=None)
    v = velocity_trajectory(16, 16, 4)
    G.set("VSTAR", v[:4])
    G.advect("VSTAR")
    G.metric_terms()
    G.adjoint("VSTAR", 0.0, 1.0)
    assert np.all(G.get("MU") == 0)
    assert np.all(G.get("Y")[1:] == 0)


def test_invalid_arguments_are_rejected():
    from paper_1608_01102_gb300 import stc
    P, G = make_pair(16, 16, N=4, precision=0)
    with pytest.raises(stc.StcError):
        stc._check(G.lib.stc_get_field(G.h, 0, 0, np.zeros(3).ctypes.data_as(stc.P_double), 3))
    with pytest.raises(stc.StcError):
        G.set_keyframes({0: (np.zeros(256), 1.0)})
    with pytest.raises(stc.StcError):
        G.project("RHO", 0, 1)
    with pytest.raises(stc.StcError):
        G.restrict(G.num_levels() - 1)
