"""Pins for the oracle's grid operators, advection, projection and metric.

Every check here compares the oracle with something other than itself: closed
forms that the discrete stencils reproduce exactly, scipy library routines,
finite differences and invariants stated by the paper (Sec. 3.1, Eq. KKTPO).
"""
import numpy as np
import pytest
import scipy.fft
import scipy.linalg
import scipy.ndimage

from oracle import advection, mac, metric, projection

pytestmark = pytest.mark.filterwarnings("ignore::DeprecationWarning")


def _grid(nx=8, ny=6):
    return mac.Grid(nx, ny, 1.0 / nx)


def _face_coords(g):
    xs = np.arange(g.nx + 1) * g.h
    ys = (np.arange(g.ny) + 0.5) * g.h
    Xx, Yx = np.meshgrid(xs, ys)
    xs = (np.arange(g.nx) + 0.5) * g.h
    ys = np.arange(g.ny + 1) * g.h
    Xy, Yy = np.meshgrid(xs, ys)
    return (Xx, Yx), (Xy, Yy)


def _centres(g):
    return np.meshgrid((np.arange(g.nx) + 0.5) * g.h, (np.arange(g.ny) + 0.5) * g.h)


# ---------------------------------------------------------------------------
# div / grad (Eq. NSA, NSB)
# ---------------------------------------------------------------------------

def test_div_of_quadratic_is_exact():
    g = _grid(8, 8)
    (Xx, Yx), (Xy, Yy) = _face_coords(g)
    vx = Xx * (1 - Xx)            # zero on the x walls
    vy = Yy * (1 - Yy) * 0.5
    d = mac.div(g, g.join(vx, vy)).reshape(g.ny, g.nx)
    X, Y = _centres(g)
    np.testing.assert_allclose(d, (1 - 2 * X) + 0.5 * (1 - 2 * Y), atol=1e-13)


def test_grad_of_quadratic_is_exact_and_zero_on_walls():
    g = _grid(8, 6)
    X, Y = _centres(g)
    p = (X ** 2 + 3 * Y ** 2).ravel()
    gx, gy = g.split(mac.grad(g, p))
    (Xx, _), (_, Yy) = _face_coords(g)
    np.testing.assert_allclose(gx[:, 1:-1], 2 * Xx[:, 1:-1], atol=1e-12)
    np.testing.assert_allclose(gy[1:-1, :], 6 * Yy[1:-1, :], atol=1e-12)
    assert np.all(gx[:, [0, -1]] == 0) and np.all(gy[[0, -1], :] == 0)


def test_grad_is_minus_div_transpose_on_closed_box():
    rng = np.random.default_rng(0)
    g = _grid(7, 5)
    m = g.interior_faces()
    v = rng.standard_normal(g.F) * m
    p = rng.standard_normal(g.C)
    assert abs(mac.grad(g, p) @ v + p @ mac.div(g, v)) < 1e-11


# ---------------------------------------------------------------------------
# Adv = (curl v) x v (Eq. NSA)
# ---------------------------------------------------------------------------

def test_vorticity_and_lamb_vector_of_solid_body_rotation():
    g = _grid(10, 10)
    (Xx, Yx), (Xy, Yy) = _face_coords(g)
    vx = -(Yx - 0.5)
    vy = (Xy - 0.5)
    v = g.join(vx, vy) * g.interior_faces()
    w = mac.vorticity(g, v).reshape(g.ny + 1, g.nx + 1)
    # interior nodes whose four faces are interior: curl of rotation = 2
    np.testing.assert_allclose(w[1:-1, 1:-1], 2.0, atol=1e-12)
    assert np.all(w[0, :] == 0) and np.all(w[:, 0] == 0)
    ax, ay = g.split(mac.adv(g, v))
    # (omega x v)_x = -omega v_y, (omega x v)_y = omega v_x, away from the walls
    np.testing.assert_allclose(ax[2:-2, 2:-2], -2.0 * (Xx[2:-2, 2:-2] - 0.5), atol=1e-12)
    np.testing.assert_allclose(ay[2:-2, 2:-2], 2.0 * -(Yy[2:-2, 2:-2] - 0.5), atol=1e-12)


def test_adv_is_zero_for_irrotational_uniform_flow():
    g = _grid(8, 8)
    vx, vy = g.split(np.zeros(g.F))
    vx[:, 1:-1] = 0.7
    v = g.join(vx, vy)
    w = mac.vorticity(g, v).reshape(g.ny + 1, g.nx + 1)
    assert np.all(w[1:-1, 1:-1] == 0)


def test_adv_jacobian_matches_central_difference():
    rng = np.random.default_rng(1)
    g = _grid(7, 6)
    m = g.interior_faces()
    v = rng.standard_normal(g.F) * m
    d = rng.standard_normal(g.F) * m
    eps = 1e-4                        # Adv is quadratic: central differences are exact
    fd = (mac.adv(g, v + eps * d) - mac.adv(g, v - eps * d)) / (2 * eps)
    np.testing.assert_allclose(mac.adv_jacobian(g, v) @ d, fd, rtol=1e-9, atol=1e-9)
    u = rng.standard_normal(g.F) * m
    np.testing.assert_allclose(mac.adv_jacobian_T_apply(g, v, u),
                               mac.adv_jacobian(g, v).T @ u, atol=1e-10)


# ---------------------------------------------------------------------------
# QUICK passive advection A(v) (Eq. Conv)
# ---------------------------------------------------------------------------

def test_quick_advection_conserves_mass_and_constants():
    rng = np.random.default_rng(2)
    g = _grid(9, 7)
    m = g.interior_faces()
    v = rng.standard_normal(g.F) * m
    A = mac.advection_matrix(g, v)
    rho = rng.random(g.C)
    assert abs((A @ rho).sum()) < 1e-12
    vs = projection.project(g, v)
    np.testing.assert_allclose(mac.advection_matrix(g, vs) @ np.full(g.C, 3.0), 0.0, atol=1e-10)


def test_quick_is_exact_for_quadratic_profiles_in_uniform_flow():
    g = _grid(12, 4)
    vx, vy = g.split(np.zeros(g.F))
    vx[:, 1:-1] = 0.8
    v = g.join(vx, vy)
    X, _ = _centres(g)
    q = lambda x: 1.0 + 2.0 * x - 3.0 * x * x
    rho = q(X).ravel()
    Arho = (mac.advection_matrix(g, v) @ rho).reshape(g.ny, g.nx)
    # cells whose upwind stencils stay clear of the walls: exact flux difference
    exact = -0.8 * (q(X + g.h / 2) - q(X - g.h / 2)) / g.h
    np.testing.assert_allclose(Arho[:, 3:-2], exact[:, 3:-2], atol=1e-11)
    # and negative flow mirrors the stencil
    vx[:, 1:-1] = -0.8
    Arho = (mac.advection_matrix(g, g.join(vx, vy)) @ rho).reshape(g.ny, g.nx)
    np.testing.assert_allclose(Arho[:, 2:-3], -exact[:, 2:-3], atol=1e-11)


def test_velocity_derivative_matches_finite_difference_and_subgradient():
    rng = np.random.default_rng(3)
    g = _grid(8, 8)
    m = g.interior_faces()
    v = (0.5 + rng.random(g.F)) * np.sign(rng.standard_normal(g.F)) * m
    x = rng.random(g.C)
    dv = rng.standard_normal(g.F) * m
    eps = 1e-6                          # no face changes sign: A is linear here
    fd = (mac.advection_matrix(g, v + eps * dv) @ x - mac.advection_matrix(g, v - eps * dv) @ x) / (2 * eps)
    np.testing.assert_allclose(mac.advection_v_derivative(g, v, x, dv), fd, atol=1e-8)
    mu = rng.standard_normal(g.C)
    assert abs(mu @ mac.advection_v_derivative(g, v, x, dv)
               - dv @ mac.advection_v_derivative_T(g, v, x, mu)) < 1e-10
    # at v = 0 the subgradient convention equals the central difference
    z = np.zeros(g.F)
    fd0 = (mac.advection_matrix(g, eps * dv) @ x - mac.advection_matrix(g, -eps * dv) @ x) / (2 * eps)
    np.testing.assert_allclose(mac.advection_v_derivative(g, z, x, dv), fd0, atol=1e-8)


# ---------------------------------------------------------------------------
# Taylor exponential and its adjoints (Eq. Adv, Eq. KKTPO)
# ---------------------------------------------------------------------------

def test_taylor_matches_expm_within_truncation_and_conserves_mass():
    rng = np.random.default_rng(4)
    g = _grid(8, 8)
    v = projection.project(g, rng.standard_normal(g.F)) * 0.6
    rho = rng.random(g.C)
    dt = 0.2
    for tol in (1e-5, 1e-10):
        out, K, terms = advection.taylor_forward(g, v, rho, dt, tol, 1.0)
        ref = scipy.linalg.expm(mac.advection_matrix(g, v).toarray() * dt) @ rho
        assert np.max(np.abs(out - ref)) < 20 * tol
        assert np.max(np.abs(terms[-1])) < tol <= np.max(np.abs(terms[-2]))
        assert abs(out.sum() - rho.sum()) < 1e-12


def test_taylor_order_limit_raises():
    rng = np.random.default_rng(5)
    g = _grid(8, 8)
    v = projection.project(g, rng.standard_normal(g.F)) * 50.0
    with pytest.raises(advection.TaylorOrderError):
        advection.taylor_forward(g, v, rng.random(g.C), 1.0, 1e-5, 1.0, kmax=8)


def test_taylor_adjoints_dot_product_and_finite_difference():
    rng = np.random.default_rng(6)
    g = _grid(8, 7)
    m = g.interior_faces()
    v = (0.4 + rng.random(g.F)) * np.sign(rng.standard_normal(g.F)) * m
    rho = rng.random(g.C)
    mu = rng.standard_normal(g.C)
    dt, K = 0.05, 6
    y = rng.standard_normal(g.C)
    lhs = mu @ advection.taylor_apply(g, v, y, dt, K)
    rhs = y @ advection.taylor_adjoint_rho(g, v, mu, dt, K)
    assert abs(lhs - rhs) < 1e-12 * max(1.0, abs(lhs))
    dv = rng.standard_normal(g.F) * m
    eps = 1e-6
    fd = mu @ (advection.taylor_apply(g, v + eps * dv, rho, dt, K)
               - advection.taylor_apply(g, v - eps * dv, rho, dt, K)) / (2 * eps)
    an = dv @ advection.taylor_adjoint_v(g, v, rho, mu, dt, K)
    assert abs(fd - an) < 1e-7 * max(1.0, abs(an))


# ---------------------------------------------------------------------------
# Projection Q (Eq. KKTPO)
# ---------------------------------------------------------------------------

def _dct_poisson(g, b):
    """Closed-form Neumann Poisson solve: the 5-point cell-centred Laplacian with
    mirror ghosts is diagonalised by the DCT-II."""
    B = scipy.fft.dctn(b.reshape(g.ny, g.nx), type=2, norm="ortho")
    kx = np.arange(g.nx)
    ky = np.arange(g.ny)
    lam = (-(4 / g.h ** 2) * np.sin(np.pi * ky / (2 * g.ny))[:, None] ** 2
           - (4 / g.h ** 2) * np.sin(np.pi * kx / (2 * g.nx))[None, :] ** 2)
    lam[0, 0] = 1.0
    P = B / lam
    P[0, 0] = 0.0
    return scipy.fft.idctn(P, type=2, norm="ortho").ravel()


@pytest.mark.parametrize("shape", [(8, 8), (16, 12), (32, 32)])
def test_projection_matches_dct_closed_form(shape):
    rng = np.random.default_rng(7)
    g = _grid(*shape)
    b = rng.standard_normal(g.C)
    b -= b.mean()
    np.testing.assert_allclose(projection.poisson_neumann(g, b), _dct_poisson(g, b), atol=1e-10)


def test_projection_properties():
    rng = np.random.default_rng(8)
    g = _grid(16, 16)
    m = g.interior_faces()
    a = rng.standard_normal(g.F) * m
    b = rng.standard_normal(g.F) * m
    Qa = projection.project(g, a)
    assert np.max(np.abs(mac.div(g, Qa))) < 1e-10
    np.testing.assert_allclose(projection.project(g, Qa), Qa, atol=1e-12)
    assert abs(Qa @ b - a @ projection.project(g, b)) < 1e-10
    phi = rng.standard_normal(g.C)
    np.testing.assert_allclose(projection.project(g, mac.grad(g, phi)), 0.0, atol=1e-10)


# ---------------------------------------------------------------------------
# Keyframe metric C_i (Sec. 4.1)
# ---------------------------------------------------------------------------

def test_metric_filters_match_scipy_gaussian_filter():
    rng = np.random.default_rng(9)
    nx, ny = 32, 24
    X = rng.random((ny, nx))
    for l in range(3):
        s = 2.0 ** l
        Mx, My = metric.blur_matrix_1d(nx, s), metric.blur_matrix_1d(ny, s)
        ref = scipy.ndimage.gaussian_filter(X, s, mode="nearest", truncate=3.0)
        np.testing.assert_allclose(My @ X @ Mx.T, ref, atol=1e-12)


def test_metric_is_symmetric_psd_and_reduces_to_identity():
    rng = np.random.default_rng(10)
    C = metric.metric_matrix(8, 8, 2)
    np.testing.assert_allclose(C, C.T, atol=1e-14)
    assert np.min(np.linalg.eigvalsh(C)) > -1e-12
    x = rng.standard_normal(64)
    np.testing.assert_allclose(metric.apply_metric(8, 8, x, 0, c=2.0), 2.0 * x)
    assert metric.default_levels(32) == 4 and metric.default_levels(128) == 6
