"""GPU parity at the benchmark's full sizes, in the launch configuration that
bench.py times (the same problem sizes, so the same kernels and launch shapes).

2D, 128^2 x 40 (the bench workload): forward advection, the backward adjoint
sweep with the 6-level metric, one SCGS sweep, the NSO residual and one STFAS
V-cycle, each against the fp64 oracle element by element.

3D, 64^3 x 60: the oracle is too slow for every output, so sampled outputs
(the first steps of the forward sweep, a few time slabs of the NSO residual)
and properties that hold at any size: mass conservation of every step, the
projection against the DCT-II closed form of the Neumann Poisson problem, and
-- on the linear problem (no Adv, no LM shift, omega = 1) -- exactness of the
last colour's local solve: after a sweep, f vanishes on every unknown of the
last colour's cells.
"""
import numpy as np
import pytest
import scipy.fft

from oracle import kkt, mac, scgs, stfas
from paper_1608_01102_gb300 import stc, workloads

from gpu_common import TOL, rel, velocity_trajectory

pytestmark = [pytest.mark.gpu, pytest.mark.filterwarnings("ignore::DeprecationWarning")]


def _pair_2d(precision=0, **over):
    cfg = workloads.config_letters(128, 40)
    star = cfg["keyframes"][40][0]
    P = kkt.Problem(128, 128, 40, 1.0 / 40, cfg["rho0"], r=1e-3, K=1.0, keyframes={40: (star, 1.0)},
                    metric_levels=6, **{k: v for k, v in over.items() if k != "scgs_omega"})
    prm = stc.default_params(128, 128, 40, precision=precision, r=1e-3, K=1.0, metric_levels=6)
    for k, v in over.items():
        setattr(prm, k, v)
    G = stc.Problem(prm, cfg["rho0"])
    G.set_keyframes({40: (star, 1.0)})
    return P, G


def test_full_2d_forward_and_adjoint_sweeps():
    P, G = _pair_2d()
    v = velocity_trajectory(128, 128, 40, amp=0.6, seed=81)
    w = workloads.random_faces(np.random.default_rng(82), 128, 128, 40, 0.1)
    G.set("VSTAR", v[:40])
    G.set("W", w)
    G.advect("VSTAR")
    G.metric_terms()
    G.adjoint("VSTAR", 1.0, 1.0 / P.K)
    rhos, Ks = kkt.forward_density(P, v[:40])
    np.testing.assert_array_equal(G.taylor_orders(), Ks)
    rho = G.get("RHO")
    for i in range(41):
        assert rel(rho[i], rhos[i]) < 1e-5, (i, rel(rho[i], rhos[i]))
    mu_ref = kkt.adjoint_density(P, v[:40], rhos, Ks)
    mu = G.get("MU")
    for s in range(40):
        assert rel(mu[s], mu_ref[s]) < 2e-5, (s, rel(mu[s], mu_ref[s]))
    dens = kkt.density_gradient(P, v[:40], rhos, Ks, mu_ref)
    y = G.get("Y")
    for s in range(1, 40):
        assert rel(y[s], w[s] - dens[s] / P.K) < 2e-5, s


def test_full_2d_sweep_residual_and_vcycle():
    P, G = _pair_2d()
    v = velocity_trajectory(128, 128, 40, amp=0.5, seed=83)
    lam = workloads.random_faces(np.random.default_rng(84), 128, 128, 40, 0.05)
    lam[0] = 0.0
    G.set("VSTAR", v[:40])
    G.set("LAMBDA", lam)
    G.prepare_targets()
    z = v[:40] - lam / P.K
    # one SCGS sweep from the zero state on the finest level
    x = kkt.zero_state(P)
    G.smooth(0, 1)
    scgs.sweep(P, P.grid, x, z, kkt.zero_state(P))
    got = G.get_state()
    for k in x:
        assert rel(got[k], x[k]) < TOL[0]["smooth"], (k, rel(got[k], x[k]))
    # the NSO residual of that state
    G.nso_residual(0)
    f = kkt.nso_residual(P, P.grid, x, z)
    r = G.get_state(prefix="RES_")
    for k in f:
        assert rel(r[k], f[k]) < 2e-5, (k, rel(r[k], f[k]))
    # one V-cycle from the zero state
    G.set_state(kkt.zero_state(P))
    x = kkt.zero_state(P)
    f_gpu = G.vcycle(1)
    f_ref = stfas.stfas_cycle(P, x, z)
    got = G.get_state()
    for k in x:
        assert rel(got[k], x[k]) < TOL[0]["vcycle"], (k, rel(got[k], x[k]))
    assert abs(f_gpu - f_ref) <= 1e-3 * f_ref


# ---------------------------------------------------------------------------
# 3D, 64^3 x 60
# ---------------------------------------------------------------------------
def _problem_3d(**over):
    cfg = workloads.config_3d(64, 60)
    prm = stc.default_params(64, 64, 60, precision=0, r=1e-3, K=1.0, metric_levels=5, nz=64)
    for k, v in over.items():
        setattr(prm, k, v)
    G = stc.Problem(prm, cfg["rho0"])
    G.set_keyframes(cfg["keyframes"])
    return cfg, G


def _velocity3(N, amp, seed):
    rng = np.random.default_rng(seed)
    m = workloads.interior_face_mask3(64, 64, 64)
    v = np.zeros((N + 1, workloads.face_count3(64, 64, 64)))
    for i in range(1, N + 1):
        c = (0.5 + 0.1 * np.sin(i), 0.5 + 0.05 * np.cos(i), 0.5)
        v[i] = workloads.swirl_velocity3(64, 64, 64, amp * (1 + 0.3 * np.sin(0.7 * i)), c, 0.3)
        v[i] += 0.02 * amp * rng.standard_normal(v.shape[1]) * m
    return v


def test_full_3d_forward_sweep_sampled_steps_and_mass():
    cfg, G = _problem_3d()
    v = _velocity3(60, 0.8, 91)
    G.set("VSTAR", v[:60])
    G.advect("VSTAR")
    rho = G.get("RHO")
    K = G.taylor_orders()
    P = kkt.Problem(64, 64, 6, 1.0 / 60, cfg["rho0"], r=1e-3, K=1.0, keyframes={}, metric_levels=0, nz=64)
    rhos, Ks = kkt.forward_density(P, v[:6])            # the first 6 steps
    np.testing.assert_array_equal(K[:6], Ks)
    for i in range(7):
        assert rel(rho[i], rhos[i]) < 1e-5, (i, rel(rho[i], rhos[i]))
    mass = rho.sum(axis=1)
    assert np.max(np.abs(mass - mass[0])) < 1e-4 * mass[0]
    assert max(K) >= 3


def _dct_poisson3(b, n, h):
    B = scipy.fft.dctn(b.reshape(n, n, n), type=2, norm="ortho")
    k = np.arange(n)
    s = (4 / h ** 2) * np.sin(np.pi * k / (2 * n)) ** 2
    lam = -(s[:, None, None] + s[None, :, None] + s[None, None, :])
    lam[0, 0, 0] = 1.0
    Pp = B / lam
    Pp[0, 0, 0] = 0.0
    return scipy.fft.idctn(Pp, type=2, norm="ortho").ravel()


def _split3(v, n):
    a, b = n * n * (n + 1), 2 * n * n * (n + 1)
    return v[:a].reshape(n, n, n + 1), v[a:b].reshape(n, n + 1, n), v[b:].reshape(n + 1, n, n)


def _div3(v, n, h):
    vx, vy, vz = _split3(v, n)
    return ((vx[:, :, 1:] - vx[:, :, :-1] + vy[:, 1:, :] - vy[:, :-1, :] + vz[1:] - vz[:-1]) / h).ravel()


def _grad3(p, n, h):
    P = p.reshape(n, n, n)
    gx = np.zeros((n, n, n + 1))
    gy = np.zeros((n, n + 1, n))
    gz = np.zeros((n + 1, n, n))
    gx[:, :, 1:n] = (P[:, :, 1:] - P[:, :, :-1]) / h
    gy[:, 1:n, :] = (P[:, 1:, :] - P[:, :-1, :]) / h
    gz[1:n] = (P[1:] - P[:-1]) / h
    return np.concatenate([gx.ravel(), gy.ravel(), gz.ravel()])


def test_full_3d_projection_against_the_dct_closed_form():
    """The AO's batched launch (60 fields at once) against Q w = w - G phi with
    phi from the DCT-II closed form of the 7-point Neumann Poisson problem
    (divergence and gradient written out with array slices here)."""
    cfg, G = _problem_3d()
    n, h = 64, 1.0 / 64
    w = workloads.random_faces3(np.random.default_rng(92), n, n, n, 60, 0.2)
    w[7] += workloads.swirl_velocity3(n, n, n, 3.0)
    G.set("W", w)
    G.project("W", 0, 60)
    out = G.get("W")
    for i in (0, 7, 31, 59):
        ref = w[i] - _grad3(_dct_poisson3(_div3(w[i], n, h), n, h), n, h)
        assert rel(out[i], ref) < 1e-4, (i, rel(out[i], ref))
        assert np.max(np.abs(_div3(out[i], n, h))) < 1e-3 * np.max(np.abs(_div3(w[i], n, h)))


def test_full_3d_nso_residual_sampled_slabs():
    cfg, G = _problem_3d()
    v = _velocity3(60, 0.5, 93)
    G.set("VSTAR", v[:60])
    G.set("LAMBDA", np.zeros_like(v[:60]))
    G.prepare_targets()
    G.smooth(0, 1)                                      # a nonzero state from the zero start
    x = G.get_state()
    G.nso_residual(0)
    r = G.get_state(prefix="RES_")
    # oracle rows of a few slabs, from a 3-step window of the state
    for t in (1, 30, 58):
        P = kkt.Problem(64, 64, 2, 1.0 / 60, cfg["rho0"], r=1e-3, K=1.0, keyframes={}, metric_levels=0, nz=64)
        xs = dict(v=x["v"][t - 1:t + 2].copy(), pbar=x["pbar"][t - 1:t + 2].copy(),
                  u=x["u"][t - 1:t + 1].copy(), p=x["p"][t - 1:t + 1].copy())
        f = kkt.nso_residual(P, P.grid, xs, v[t - 1:t + 1])
        # window slab 1 is global slab t: rows 1, 2 at v_t / pbar_t, rows 3, 4 at u_t / p_{t+1}
        assert rel(r["v"][t], f["v"][1]) < 2e-5, t
        assert rel(r["pbar"][t], f["pbar"][1]) < 2e-5, t
        assert rel(r["u"][t], f["u"][1]) < 2e-5, t
        assert rel(r["p"][t], f["p"][1]) < 2e-5, t


def test_full_3d_linear_sweep_solves_the_last_colour_exactly():
    """64^3 x 60 through the thread-per-cell kernel: on the linear problem with
    the exact local Jacobian (no Adv, no LM shift, omega = 1) the update of the
    last colour (7) zeroes f on all its cells' unknowns."""
    cfg, G = _problem_3d(self_advection=0, lm_shift=0.0, scgs_omega=1.0)
    v = _velocity3(60, 0.5, 94)
    G.set("VSTAR", v[:60])
    G.set("LAMBDA", np.zeros_like(v[:60]))
    G.prepare_targets()
    f0 = G.nso_residual(0)
    G.smooth(0, 1)
    G.nso_residual(0)
    r = G.get_state(prefix="RES_")
    g = mac.Grid3(64, 64, 64, 1.0 / 64)
    idx = scgs.colour_cells(g, 7)
    faces, active = scgs.cell_faces(g, idx)
    fl = faces[active > 0]
    cells = g.cell(*idx)
    local = max(np.max(np.abs(r["v"][1:, fl])), np.max(np.abs(r["u"][:, fl])),
                np.max(np.abs(r["pbar"][1:, cells])), np.max(np.abs(r["p"][:, cells])))
    assert local < 1e-3 * f0, (local, f0)
    everywhere = max(np.max(np.abs(r[k])) for k in r)
    assert everywhere > 10 * local                       # the other colours' rows are not zero


def test_full_3d_grid_vcycle_against_the_oracle_two_steps():
    """One V(2,2)-cycle on the full 64^3 grid (5 levels; the finest level's
    colours run the thread-per-cell SCGS and the two-pass residual) restricted
    to 2 timesteps, with Adv and the default safeguards, from the zero state
    toward a smooth target, against the oracle's cycle (~20-40 s of CPU)."""
    n, N = 64, 2
    cfg = workloads.config_3d(64, 60)
    prm = stc.default_params(n, n, N, precision=0, r=1e-3, K=1.0, metric_levels=0, nz=n, dt=1.0 / 60)
    G = stc.Problem(prm, cfg["rho0"])
    P = kkt.Problem(n, n, N, 1.0 / 60, cfg["rho0"], r=1e-3, K=1.0, metric_levels=0, nz=n)
    z = np.zeros((N, P.grid.F))
    z[1] = workloads.swirl_velocity3(n, n, n, 0.5)
    G.set("VSTAR", z)
    G.set("LAMBDA", np.zeros_like(z))
    G.prepare_targets()
    x = kkt.zero_state(P)
    f_gpu = G.vcycle(1)
    f_ref = stfas.stfas_cycle(P, x, z)
    got = G.get_state(0)
    for k in x:
        assert rel(got[k], x[k]) < TOL[0]["vcycle"], (k, rel(got[k], x[k]))
    assert abs(f_gpu - f_ref) <= 1e-3 * f_ref
    G.close()
