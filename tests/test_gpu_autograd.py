"""GPU: the forward simulation as a torch.autograd.Function (the differentiable
simulation) against the fp64 oracle.

The oracle solves each implicit Navier-Stokes step exactly (Newton, sparse
direct solves; oracle.brute) and differentiates the whole chain by its own
adjoint; the library iterates Picard with its multigrid projection, so the
two agree to the projection's truncation.  Also checked: central differences
of the library's own map, and that segment checkpointing changes nothing.
"""
import numpy as np
import pytest

from oracle import brute, kkt, projection
from paper_1608_01102_gb300 import workloads

pytestmark = [pytest.mark.gpu, pytest.mark.filterwarnings("ignore::DeprecationWarning")]

torch = pytest.importorskip("torch")


def _case(nz, precision, checkpoint_every=None, N=6):
    from paper_1608_01102_gb300 import autograd
    if nz:
        n = 8
        rho0 = workloads.gaussian_ball3(n, n, nz, (0.5, 0.35, 0.5), 0.15)
        star = workloads.gaussian_ball3(n, n, nz, (0.5, 0.6, 0.45), 0.15)
        rng = np.random.default_rng(51)
        u = workloads.random_faces3(rng, n, n, nz, N, 0.1) + workloads.swirl_velocity3(n, n, nz, 2.0)[None]
    else:
        n = 16
        rho0 = workloads.gaussian_ball(n, n, (0.5, 0.35), 0.12)
        star = workloads.gaussian_ball(n, n, (0.5, 0.6), 0.12)
        rng = np.random.default_rng(52)
        u = workloads.random_faces(rng, n, n, N, 0.1) + workloads.swirl_velocity(n, n, 2.0)[None]
    P = kkt.Problem(n, n, N, 1.0 / N, rho0, r=1e-30, K=1.0, keyframes={N: (star, 1.0)}, metric_levels=0,
                    nz=nz)
    u = u * P.grid.interior_faces()
    sim = autograd.Simulation(n, n, N, rho0, nz=nz, precision=precision, checkpoint_every=checkpoint_every)
    return P, sim, u, star


def _loss_and_grad(sim, u, star):
    from paper_1608_01102_gb300 import autograd
    ut = torch.tensor(u, dtype=sim.dtype, device="cuda", requires_grad=True)
    rho = autograd.simulate(ut, sim)
    st = torch.tensor(star, dtype=sim.dtype, device="cuda")
    loss = 0.5 * ((rho[-1] - st) ** 2).sum()
    loss.backward()
    return float(loss.detach()), ut.grad.detach().cpu().double().numpy(), rho.detach().cpu().double().numpy()


@pytest.mark.parametrize("nz", [0, 8])
@pytest.mark.parametrize("precision", [1, 0])
def test_forward_and_gradient_match_the_oracle(nz, precision):
    P, sim, u, star = _case(nz, precision)
    loss, g, rho = _loss_and_grad(sim, u, star)
    v_ref = brute.simulate(P, u)
    rho_ref, _ = kkt.forward_density(P, v_ref)
    J_ref, g_ref = brute.objective_and_gradient(P, u)
    tol_f = 1e-6 if precision == 1 else 1e-4
    tol_g = 1e-5 if precision == 1 else 2e-3
    for i in range(P.N + 1):
        assert np.linalg.norm(rho[i] - rho_ref[i]) <= tol_f * np.linalg.norm(rho_ref[i]), i
    assert abs(loss - J_ref) <= tol_f * 10 * J_ref
    m = P.grid.interior_faces()
    err = np.linalg.norm((g - g_ref) * m) / np.linalg.norm(g_ref * m)
    assert err < tol_g, err
    assert np.max(np.abs(rho[-1] - P.rho0)) > 1e-2        # the forces do move the density
    sim.close()


@pytest.mark.parametrize("nz", [0, 8])
def test_gradient_matches_central_differences(nz):
    P, sim, u, star = _case(nz, 1)
    _, g, _ = _loss_and_grad(sim, u, star)
    rng = np.random.default_rng(53)
    for _ in range(3):
        d = rng.standard_normal(u.shape) * P.grid.interior_faces()
        eps = 1e-5
        lp = _loss_and_grad(sim, u + eps * d, star)[0]
        lm = _loss_and_grad(sim, u - eps * d, star)[0]
        fd = (lp - lm) / (2 * eps)
        an = float(np.sum(g * d))
        assert abs(fd - an) <= 1e-5 * max(abs(an), 1e-12), (fd, an)
    sim.close()


@pytest.mark.parametrize("nz", [0, 8])
def test_checkpointed_segments_give_the_same_gradient(nz):
    P, sim, u, star = _case(nz, 1)
    l1, g1, r1 = _loss_and_grad(sim, u, star)
    sim.close()
    _, simc, _, _ = _case(nz, 1, checkpoint_every=2)
    l2, g2, r2 = _loss_and_grad(simc, u, star)
    assert len(simc.segments) == 3
    assert abs(l1 - l2) <= 1e-12 * abs(l1)
    np.testing.assert_allclose(r2, r1, rtol=0, atol=1e-12 * np.max(np.abs(r1)))
    assert np.linalg.norm(g2 - g1) <= 1e-9 * np.linalg.norm(g1)
    simc.close()


def test_full_size_gradient_against_central_differences_128cubed():
    """The differentiable-simulation workload at size: 128^3 cells, 48 steps,
    fp32, checkpoint-and-recompute every 8 steps, smooth seeded random forces
    (correlation length 8 cells, max |u| = 0.1), loss 1/2 ||rho_N - rho*||^2 to
    a blurred ellipsoid union.  The gradient from the adjoint backward pass
    against central differences of the same map on 16 seeded random
    directions (each a smooth random field like u times seeded per-step
    weights, so that the differences stay where the map is smooth); the
    checkpointed forward pass keeps 6 segment starts instead of 48 steps."""
    from paper_1608_01102_gb300 import autograd
    cfg = workloads.config_autograd(128, 48)
    n, N = 128, 48
    sim = autograd.Simulation(n, n, N, cfg["rho0"], nz=n, precision=0, checkpoint_every=8)
    assert len(sim.segments) == 6
    u = cfg["u"]
    loss, g, rho = _loss_and_grad(sim, u, cfg["star"])
    assert np.isfinite(loss) and np.all(np.isfinite(g))
    assert np.max(np.abs(rho[-1] - cfg["rho0"])) > 1e-3       # the forces move the density
    errs = []
    for k in range(16):
        f = workloads.gaussian_random_faces3(n, n, n, 1, 7000 + k, 8.0, 0.1)[0]
        d = np.random.default_rng(7100 + k).standard_normal(N)[:, None] * f[None]
        eps = 0.05
        lp = _loss_and_grad_value(sim, u + eps * d, cfg["star"])
        lm = _loss_and_grad_value(sim, u - eps * d, cfg["star"])
        fd = (lp - lm) / (2 * eps)
        an = float(np.sum(g * d))
        errs.append(abs(fd - an) / max(abs(an), 1e-30))
    errs = np.array(errs)
    assert np.median(errs) < 1e-2 and np.max(errs) < 5e-2, errs
    sim.close()


def _loss_and_grad_value(sim, u, star):
    from paper_1608_01102_gb300 import autograd
    with torch.no_grad():
        ut = torch.tensor(u, dtype=sim.dtype, device="cuda")
        rho = autograd.simulate(ut, sim)
        st = torch.tensor(star, dtype=sim.dtype, device="cuda")
        return float(0.5 * ((rho[-1] - st) ** 2).sum())


GOLDEN32 = __import__("os").path.join(__import__("os").path.dirname(__import__("os").path.abspath(__file__)),
                                      "golden", "autograd_32cubed.npz")


@pytest.mark.parametrize("precision", [1, 0])
def test_gradient_matches_the_oracle_at_32cubed(precision):
    """The autograd map at 32^3 (the differentiable-simulation recipe, 2 steps
    of dt = 1/48) against the fp64 oracle's Newton-solved chain and adjoint
    (tests/golden/make_autograd_32.py): the loss, ||g|| and g's projections
    on 32 seeded random directions.  For an error e of g, a projection on a
    direction of independent unit normals is distributed as N(0, ||e||^2), so
    each projection must agree within 4 tol ||g||."""
    import os
    from paper_1608_01102_gb300 import autograd
    if not os.path.exists(GOLDEN32):
        pytest.skip("tests/golden/autograd_32cubed.npz has not been written")
    ref = np.load(GOLDEN32)
    n, N = 32, 2
    cfg = workloads.config_autograd(n, N)
    sim = autograd.Simulation(n, n, N, cfg["rho0"], nz=n, dt=1.0 / 48, precision=precision)
    m = workloads.interior_face_mask3(n, n, n)
    loss, g, _ = _loss_and_grad(sim, cfg["u"] * m, cfg["star"])
    tol = 1e-5 if precision == 1 else 2e-3
    gn = float(ref["gnorm"])
    assert abs(loss - float(ref["loss"])) <= tol * float(ref["loss"])
    assert abs(np.linalg.norm(g * m) - gn) <= tol * gn
    for k in range(len(ref["proj"])):
        d = np.random.default_rng(9000 + k).standard_normal(g.shape) * m
        assert abs(float(np.sum(g * d)) - float(ref["proj"][k])) <= 4 * tol * gn, k
    sim.close()
