"""Pins for the oracle's 3D path (the method on an n^3 grid, Sec. 3.1 with a
third axis).

References: the 2D oracle (pinned in test_oracle_operators / test_oracle_solver)
on fields that do not vary along one axis and have no velocity along it -- on
each of the three coordinate planes the 3D curl, Lamb vector and QUICK flux
reduce to the 2D ones; closed forms (linear fields through the transfers, the
DCT-II Neumann Poisson solve, solid-body rotation); finite differences; the
zero-control special case; dense and least-squares library solves.
"""
import numpy as np
import pytest
import scipy.fft

from oracle import admm, brute, kkt, mac, metric, projection, scgs, stfas
from paper_1608_01102_gb300 import workloads

pytestmark = pytest.mark.filterwarnings("ignore::DeprecationWarning")


def _embed_plane(g3, g2, w2, plane):
    """3D face field constant along the axis normal to ``plane`` with zero
    velocity along it, from a 2D face field w2 on g2.

    plane 'xy': 2D (x, y) = 3D (x, y); 'yz': 2D (x, y) = 3D (y, z);
    'zx': 2D (x, y) = 3D (z, x).  (Each is a cyclic relabelling of the axes,
    so orientation -- the sign of the curl -- is kept.)"""
    a, b = g2.split(w2)          # a: 2D x-faces (ny2, nx2+1); b: 2D y-faces (ny2+1, nx2)
    nx, ny, nz = g3.nx, g3.ny, g3.nz
    zx, zy, zz = (np.zeros(s) for s in g3.face_shapes())
    if plane == "xy":
        zx[:] = a[None]
        zy[:] = b[None]
    elif plane == "yz":          # 2D x = 3D y (index j), 2D y = 3D z (index k)
        zy[:] = a[:, :, None]
        zz[:] = b[:, :, None]
    else:                        # 2D x = 3D z (index k), 2D y = 3D x (index i)
        zz[:] = a.T[:, None, :]
        zx[:] = b.T[:, None, :]
    return g3.join(zx, zy, zz)


def _plane_view(g3, f3, plane):
    """(2D x-component, 2D y-component, normal component) of a 3D face field
    taken on the first slab along the plane's normal axis."""
    fx, fy, fz = g3.split(f3)
    if plane == "xy":
        return fx[0], fy[0], fz
    if plane == "yz":
        return fy[:, :, 0], fz[:, :, 0], fx
    return fz[:, 0, :].T, fx[:, 0, :].T, fy


_PLANE_DIMS = {"xy": lambda nx, ny, nz: (nx, ny), "yz": lambda nx, ny, nz: (ny, nz),
               "zx": lambda nx, ny, nz: (nz, nx)}


@pytest.mark.parametrize("plane", ["xy", "yz", "zx"])
def test_lamb_vector_reduces_to_2d_on_each_plane(plane):
    rng = np.random.default_rng(31)
    nx, ny, nz = 6, 5, 4
    h = 1.0 / nx
    g3 = mac.Grid3(nx, ny, nz, h)
    g2 = mac.Grid(*_PLANE_DIMS[plane](nx, ny, nz), h)
    w2 = rng.standard_normal(g2.F) * g2.interior_faces()
    v3 = _embed_plane(g3, g2, w2, plane)
    a2x, a2y = g2.split(mac.adv(g2, w2))
    ax, ay, an = _plane_view(g3, mac.adv(g3, v3), plane)
    np.testing.assert_allclose(ax, a2x, atol=1e-13)
    np.testing.assert_allclose(ay, a2y, atol=1e-13)
    assert np.max(np.abs(an)) == 0.0
    # the Jacobian transpose through the same embedding
    u2 = rng.standard_normal(g2.F) * g2.interior_faces()
    u3 = _embed_plane(g3, g2, u2, plane)
    t2x, t2y = g2.split(mac.adv_jacobian_T_apply(g2, w2, u2))
    tx, ty, _ = _plane_view(g3, mac.adv_jacobian_T_apply(g3, v3, u3), plane)
    # u3 is constant along the normal axis, so each slab's transposed stencil
    # gathers exactly the 2D contributions
    np.testing.assert_allclose(tx, t2x, atol=1e-12)
    np.testing.assert_allclose(ty, t2y, atol=1e-12)


@pytest.mark.parametrize("plane", ["xy", "yz", "zx"])
def test_quick_advection_reduces_to_2d_on_each_plane(plane):
    rng = np.random.default_rng(32)
    nx, ny, nz = 6, 5, 4
    h = 1.0 / nx
    g3 = mac.Grid3(nx, ny, nz, h)
    d2 = _PLANE_DIMS[plane](nx, ny, nz)
    g2 = mac.Grid(*d2, h)
    w2 = rng.standard_normal(g2.F) * g2.interior_faces()
    v3 = _embed_plane(g3, g2, w2, plane)
    r2 = rng.random(g2.C).reshape(d2[1], d2[0])        # (2D y, 2D x)
    if plane == "xy":
        r3 = np.repeat(r2[None], nz, 0)
    elif plane == "yz":
        r3 = np.repeat(r2[:, :, None], nx, 2)           # (k=2D y, j=2D x, i)
    else:
        r3 = np.repeat(r2.T[:, None, :], ny, 1)         # (k=2D x, j, i=2D y)
    A3 = (mac.advection_matrix(g3, v3) @ r3.ravel()).reshape(g3.cell_shape())
    A2 = (mac.advection_matrix(g2, w2) @ r2.ravel()).reshape(d2[1], d2[0])
    got = {"xy": A3[0], "yz": A3[:, :, 0], "zx": A3[:, 0, :].T}[plane]
    np.testing.assert_allclose(got, A2, atol=1e-12)


def test_curl_and_lamb_vector_of_solid_body_rotation():
    """v = (-(y - 1/2), x - 1/2, 0): omega = (0, 0, 2) on interior edges and
    (omega x v) = -2 (x - 1/2, y - 1/2, 0) on faces whose stencils avoid the walls."""
    n = 8
    g = mac.Grid3(n, n, n, 1.0 / n)
    h = g.h
    comps = []
    for axis in range(3):
        shp = g.face_shapes()[axis]
        ax = [np.arange(m) * h if a == 2 - axis else (np.arange(m) + 0.5) * h
              for a, m in enumerate(shp)]
        Z, Y, X = np.meshgrid(*ax, indexing="ij")
        comps.append([-(Y - 0.5), X - 0.5, 0 * X][axis])
    v = g.join(*comps) * g.interior_faces()
    wx, wy, wz = mac.vorticity(g, v)
    Wz = wz.reshape(n, n + 1, n + 1)
    np.testing.assert_allclose(Wz[:, 1:n, 1:n], 2.0, atol=1e-12)
    assert np.max(np.abs(wx)) < 1e-12 and np.max(np.abs(wy)) < 1e-12
    ax_, ay_, az_ = g.split(mac.adv(g, v))
    X = np.arange(n + 1) * h
    Yc = (np.arange(n) + 0.5) * h
    want_x = -2.0 * (X[None, None, :] - 0.5) + 0 * Yc[None, :, None]
    np.testing.assert_allclose(ax_[:, 2:n - 2, 2:n - 1], want_x[:, 2:n - 2, 2:n - 1] * np.ones((n, 1, 1)),
                               atol=1e-12)
    assert np.max(np.abs(az_)) < 1e-12


def test_adv_jacobian_and_transpose_3d():
    rng = np.random.default_rng(33)
    g = mac.Grid3(5, 4, 3, 0.2)
    m = g.interior_faces()
    v = rng.standard_normal(g.F) * m
    d = rng.standard_normal(g.F) * m
    u = rng.standard_normal(g.F)
    J = mac.adv_jacobian(g, v)
    eps = 1e-6
    fd = (mac.adv(g, v + eps * d) - mac.adv(g, v - eps * d)) / (2 * eps)
    np.testing.assert_allclose(J @ d, fd, atol=1e-8)
    assert abs(u @ (J @ d) - d @ mac.adv_jacobian_T_apply(g, v, u)) < 1e-11


def test_grad_is_minus_div_transpose_and_quick_conserves_mass_3d():
    rng = np.random.default_rng(34)
    g = mac.Grid3(5, 4, 6, 0.2)
    o = mac.ops(g)
    m = g.interior_faces()
    # closed box: G = -D^T on interior faces, zero rows on walls
    np.testing.assert_allclose(o["G"].toarray(), -(o["D"].T.toarray() * m[:, None]), atol=1e-12)
    v = rng.standard_normal(g.F) * g.interior_faces()
    A = mac.advection_matrix(g, v)
    np.testing.assert_allclose(np.ones(g.C) @ A, 0.0, atol=1e-11)
    np.testing.assert_allclose(A @ np.ones(g.C), -mac.div(g, v), atol=1e-11)


def test_velocity_derivative_matches_finite_difference_3d():
    rng = np.random.default_rng(35)
    g = mac.Grid3(5, 5, 4, 0.2)
    m = g.interior_faces()
    v = rng.standard_normal(g.F)
    v = np.where(np.abs(v) < 0.05, 0.3, v) * m     # interior faces away from the upwind switch
    x = rng.random(g.C)
    mu = rng.standard_normal(g.C)
    d = rng.standard_normal(g.F) * m
    eps = 1e-7
    fd = mu @ ((mac.advection_matrix(g, v + eps * d) - mac.advection_matrix(g, v - eps * d)) @ x) / (2 * eps)
    assert abs(fd - d @ mac.advection_v_derivative_T(g, v, x, mu)) < 1e-7 * max(1.0, abs(fd))


def _dct_poisson3(g, b):
    """Closed-form 3D Neumann Poisson solve (7-point Laplacian, DCT-II)."""
    B = scipy.fft.dctn(b.reshape(g.cell_shape()), type=2, norm="ortho")
    lam = 0.0
    for axis, n in enumerate(g.cell_shape()):
        k = np.arange(n)
        shape = [1, 1, 1]
        shape[axis] = n
        lam = lam - (4 / g.h ** 2) * (np.sin(np.pi * k / (2 * n)) ** 2).reshape(shape)
    lam = np.broadcast_to(lam, B.shape).copy()
    lam[0, 0, 0] = 1.0
    P = B / lam
    P[0, 0, 0] = 0.0
    return scipy.fft.idctn(P, type=2, norm="ortho").ravel()


def test_projection_matches_dct_closed_form_and_is_solenoidal_3d():
    rng = np.random.default_rng(36)
    g = mac.Grid3(8, 6, 4, 1.0 / 8)
    b = rng.standard_normal(g.C)
    b -= b.mean()
    np.testing.assert_allclose(projection.poisson_neumann(g, b), _dct_poisson3(g, b), atol=1e-10)
    a = rng.standard_normal(g.F) * g.interior_faces()
    Qa = projection.project(g, a)
    assert np.max(np.abs(mac.div(g, Qa))) < 1e-10
    np.testing.assert_allclose(projection.project(g, Qa), Qa, atol=1e-12)


def test_metric_3d_is_separable_blur_and_symmetric():
    rng = np.random.default_rng(37)
    nx, ny, nz = 6, 5, 4
    X = rng.random((nz, ny, nx))
    C = metric.metric_matrix(nx, ny, 2, nz=nz)
    np.testing.assert_allclose(C, C.T, atol=1e-13)
    # one level: G^T G x with G the Kronecker product of the axis blurs
    Mz, My, Mx = (metric.blur_matrix_1d(n, 1.0) for n in (nz, ny, nx))
    G = np.kron(Mz, np.kron(My, Mx))
    np.testing.assert_allclose(metric.apply_metric(nx, ny, X.ravel(), 1, nz=nz),
                               G.T @ (G @ X.ravel()), atol=1e-13)


def test_transfers_3d_closed_forms():
    """R of a linear cell field is the coarse linear field; P of a linear field
    is linear away from the clamped walls; faces likewise per component."""
    f = mac.Grid3(8, 6, 4, 1.0 / 8)
    c = f.coarse()

    def lin(X, Y, Z):
        return X + 2 * Y - 3 * Z

    def centres(g):
        Z, Y, X = np.meshgrid(*((np.arange(n) + .5) * g.h for n in g.cell_shape()), indexing="ij")
        return X, Y, Z

    def face_pos(g, axis):
        shp = g.face_shapes()[axis]
        ax = [np.arange(m) * g.h if a == 2 - axis else (np.arange(m) + .5) * g.h
              for a, m in enumerate(shp)]
        Z, Y, X = np.meshgrid(*ax, indexing="ij")
        return X, Y, Z

    np.testing.assert_allclose(stfas.restrict_cells(f, lin(*centres(f)).ravel()),
                               lin(*centres(c)).ravel(), atol=1e-13)
    p = stfas.prolong_cells(f, c, lin(*centres(c)).ravel()).reshape(f.cell_shape())
    np.testing.assert_allclose(p[1:-1, 1:-1, 1:-1], lin(*centres(f))[1:-1, 1:-1, 1:-1], atol=1e-13)
    for axis in range(3):
        vc = [np.zeros(s) for s in c.face_shapes()]
        vf = [np.zeros(s) for s in f.face_shapes()]
        vc[axis] = lin(*face_pos(c, axis))
        vf[axis] = lin(*face_pos(f, axis))
        pf = f.split(stfas.prolong_faces(f, c, c.join(*vc)))
        np.testing.assert_allclose(pf[axis][1:-1, 1:-1, 1:-1], vf[axis][1:-1, 1:-1, 1:-1], atol=1e-13)
        rc = c.split(stfas.restrict_faces(f, f.join(*vf)))
        np.testing.assert_allclose(rc[axis], vc[axis], atol=1e-13)
        for other in range(3):
            if other != axis:
                assert np.max(np.abs(pf[other])) == 0.0 and np.max(np.abs(rc[other])) == 0.0
    # R and P are adjoint up to the volume ratio on cells: <R a, b>_c 2^3 = <a, P' b>
    rng = np.random.default_rng(38)
    a = rng.standard_normal(f.C)
    assert abs(np.sum(stfas.restrict_cells(f, a)) * 8 - np.sum(a)) < 1e-10


def _problem3(n=4, N=3, levels=1, **kw):
    rho0 = workloads.gaussian_ball3(n, n, n, (0.5, 0.35, 0.5), 0.2)
    star = workloads.gaussian_ball3(n, n, n, (0.5, 0.65, 0.45), 0.2)
    args = dict(r=1e-2, K=1.0, keyframes={N: (star, 1.0)}, metric_levels=levels, nz=n)
    args.update(kw)
    return kkt.Problem(n, n, N, 1.0 / N, rho0, **args)


def _solenoidal(P, rng, scale):
    v = np.zeros((P.N + 1, P.grid.F))
    for i in range(1, P.N + 1):
        v[i] = projection.project(P.grid, rng.standard_normal(P.grid.F)) * scale
    return v


def test_full_resimulation_gradient_matches_central_differences_6x6x6x3():
    """brute.objective_and_gradient on the 3D grid (Newton-solved implicit
    steps and their adjoint) against central differences of J(u)."""
    from oracle import brute, mac
    rng = np.random.default_rng(47)
    P = _problem3(n=6, N=3, r=0.05)
    m = mac.ops(P.grid)["mask"]
    u = rng.standard_normal((P.N, P.grid.F)) * m * 0.3
    J, g = brute.objective_and_gradient(P, u)

    def Jf(uu, Ks):
        rhos, _ = kkt.forward_density(P, brute.simulate(P, uu), Ks)
        return 0.5 * P.r * float(np.sum(uu * uu)) + P.misfit(rhos)

    _, Ks = kkt.forward_density(P, brute.simulate(P, u))
    assert abs(J - Jf(u, Ks)) <= 1e-12 * abs(J)
    for _ in range(2):
        d = rng.standard_normal(u.shape) * m
        eps = 1e-5
        fd = (Jf(u + eps * d, Ks) - Jf(u - eps * d, Ks)) / (2 * eps)
        an = float(np.sum(g * d))
        assert abs(fd - an) <= 1e-6 * max(abs(an), 1e-12), (fd, an)


def test_reduced_gradient_matches_central_differences_3d():
    rng = np.random.default_rng(39)
    P = _problem3(levels=1)
    v = _solenoidal(P, rng, 0.4)
    _, Ks = kkt.forward_density(P, v)
    g = kkt.reduced_gradient(P, v)
    for _ in range(2):
        d = _solenoidal(P, rng, 1.0)
        eps = 1e-6
        fd = (kkt.objective(P, v + eps * d, Ks) - kkt.objective(P, v - eps * d, Ks)) / (2 * eps)
        an = float(np.sum(g * d))
        assert abs(fd - an) <= 1e-6 * max(abs(an), 1e-12), (fd, an)


def test_zero_control_gives_zero_gradient_and_residual_3d():
    n, N = 4, 3
    P = _problem3(n, N)
    P.v0 = projection.project(P.grid, workloads.swirl_velocity3(n, n, n, 2.0))
    v = np.zeros((N + 1, P.grid.F))
    u = np.zeros((N, P.grid.F))
    p = np.zeros((N, P.grid.C))
    v[0] = P.v0
    for i in range(N):
        v[i + 1], p[i] = brute.ns_step(P.grid, v[i], u[i], P.dt)
    rhos, _ = kkt.forward_density(P, v)
    P.keyframes = {N: (rhos[N].copy(), 1.0)}
    assert np.max(np.abs(kkt.reduced_gradient(P, v))) < 1e-9
    assert np.max(np.abs(rhos[N] - P.rho0)) > 1e-3
    x = dict(v=v, pbar=np.zeros((N + 1, P.grid.C)), u=u, p=p)
    assert kkt.state_inf(kkt.nso_residual(P, P.grid, x, v[:N].copy())) < 1e-9


def _random_state(P, rng):
    m = P.grid.interior_faces()
    x = dict(v=rng.standard_normal((P.N + 1, P.grid.F)) * m,
             pbar=rng.standard_normal((P.N + 1, P.grid.C)),
             u=rng.standard_normal((P.N, P.grid.F)) * m,
             p=rng.standard_normal((P.N, P.grid.C)))
    x["v"][0] = 0.0
    x["pbar"][0] = 0.0
    return x


def test_nso_residual_is_gradient_of_potential_3d():
    rng = np.random.default_rng(40)
    P = _problem3(4, 2)
    x = _random_state(P, rng)
    z = rng.standard_normal((P.N, P.grid.F)) * P.grid.interior_faces()
    f = kkt.nso_residual(P, P.grid, x, z)
    for _ in range(2):
        d = _random_state(P, rng)
        eps = 1e-6
        xp = {k: x[k] + eps * d[k] for k in x}
        xm = {k: x[k] - eps * d[k] for k in x}
        fd = (kkt.nso_potential(P, P.grid, xp, z) - kkt.nso_potential(P, P.grid, xm, z)) / (2 * eps)
        an = sum(float(np.sum(f[k] * d[k])) for k in f)
        assert abs(fd - an) <= 1e-7 * abs(an)


def test_block_thomas_equals_dense_solve_and_blocks_are_the_jacobian_3d():
    rng = np.random.default_rng(41)
    P = _problem3(4, 3, lm_shift=0.0)
    x = _random_state(P, rng)
    faces, active = scgs.cell_faces(P.grid, scgs.colour_cells(P.grid, 5))
    Dg, Lo, Up = scgs.assemble(P, P.grid, x, faces, active)
    assert Dg.shape[2:] == (7, 7)
    b = rng.standard_normal((faces.shape[0], 2 * P.N, 7))
    sol = scgs.block_thomas(Dg, Lo, Up, b)
    for c in range(faces.shape[0]):
        A = scgs.dense_from_blocks(Dg[c], Lo[c], Up[c])
        np.testing.assert_allclose(sol[c].ravel(), np.linalg.solve(A, b[c].ravel()), rtol=1e-9, atol=1e-9)
    # with u = 0 the blocks of an interior cell are finite-difference columns of f
    x["u"][:] = 0.0
    g = P.grid
    idx = (np.array([1]), np.array([2]), np.array([1]))
    faces, active = scgs.cell_faces(g, idx)
    assert np.all(active == 1.0)
    cell = g.cell(*idx)[0]
    Dg, Lo, Up = scgs.assemble(P, g, x, faces, active)
    A = scgs.dense_from_blocks(Dg[0], Lo[0], Up[0])
    z = np.zeros((P.N, g.F))
    unk = []
    for i in range(P.N):
        unk += [("u", i, f) for f in faces[0]] + [("p", i, cell)]
        unk += [("v", i + 1, f) for f in faces[0]] + [("pbar", i + 1, cell)]
    f0 = kkt.nso_residual(P, g, x, z)
    eps = 1e-6
    for col, (k, i, ix) in enumerate(unk):
        xp = kkt.copy_state(x)
        xp[k][i][ix] += eps
        fp = kkt.nso_residual(P, g, xp, z)
        fd = np.array([(fp[kk][ii][jx] - f0[kk][ii][jx]) / eps for kk, ii, jx in unk])
        np.testing.assert_allclose(A[:, col], fd, atol=2e-4 * max(1.0, np.max(np.abs(fd))))


def _linear_solution(P, z):
    g = P.grid
    m = g.interior_faces().astype(bool)
    fi = np.flatnonzero(m)
    layout = ([("v", i, fi) for i in range(1, P.N + 1)] + [("pbar", i, np.arange(g.C)) for i in range(1, P.N + 1)] +
              [("u", i, fi) for i in range(P.N)] + [("p", i, np.arange(g.C)) for i in range(P.N)])

    def flat(s):
        return np.concatenate([s[k][i][ix] for k, i, ix in layout])

    def unflat(vec):
        s = kkt.zero_state(P)
        o = 0
        for k, i, ix in layout:
            s[k][i][ix] = vec[o:o + ix.size]
            o += ix.size
        return s

    n = sum(ix.size for _, _, ix in layout)
    b0 = flat(kkt.nso_residual(P, g, unflat(np.zeros(n)), z))
    A = np.zeros((n, n))
    for k in range(n):
        e = np.zeros(n)
        e[k] = 1.0
        A[:, k] = flat(kkt.nso_residual(P, g, unflat(e), z)) - b0
    return unflat(np.linalg.lstsq(A, -b0, rcond=None)[0])


def test_vcycles_converge_to_direct_solution_of_linear_saddle_problem_3d():
    """Non-cubic 6 x 6 x 4 grid (levels 6x6x4 -> 3x3x2), 2 steps, no Adv."""
    rng = np.random.default_rng(42)
    nx, nz, N = 6, 4, 2
    rho0 = workloads.gaussian_ball3(nx, nx, nz, (0.5, 0.35, 0.3), 0.2)
    P = kkt.Problem(nx, nx, N, 1.0 / N, rho0, r=1e-2, K=1.0, nz=nz, coarsest_n=2,
                    self_advection=False, keyframes={N: (rho0, 1.0)})
    assert [(g.nx, g.ny, g.nz) for g in stfas.hierarchy(P)] == [(6, 6, 4), (3, 3, 2)]
    z = np.array([projection.project(P.grid, w) for w in workloads.random_faces3(rng, nx, nx, nz, N)])
    ref = _linear_solution(P, z)
    x = kkt.zero_state(P)
    hist = [stfas.stfas_cycle(P, x, z) for _ in range(20)]
    for k in ("v", "u", "pbar", "p"):
        scale = max(np.max(np.abs(ref[k])), 1e-3 * np.max(np.abs(ref["u"])))
        np.testing.assert_allclose(x[k], ref[k], atol=1e-7 * scale)
    assert max(hist[k + 1] / hist[k] for k in range(1, 8)) < 0.35


def test_admm_decreases_the_objective_3d():
    """A few ADMM iterations on a tiny 3D problem lower J and keep v solenoidal."""
    P = _problem3(4, 3, levels=1, r=1e-2)
    J0 = kkt.objective(P, np.zeros((P.N + 1, P.grid.F)))
    x, vstar, lam, hist = admm.solve(P, tol=1e-12, max_admm=6, eps_admm=0.0)
    J = kkt.objective(P, x["v"])
    assert J < 0.9 * J0, (J, J0)
    assert max(np.max(np.abs(mac.div(P.grid, a))) for a in x["v"]) < 1e-6
    assert hist[-1]["kkt_rel"] < hist[0]["kkt_rel"]


# ---------------------------------------------------------------------------
# periodic boundaries (every axis wraps; the paper's periodic benchmarks are 3D)
# ---------------------------------------------------------------------------
def _roll(g, v, axis, sh):
    """Periodic shift of a face field by sh cells along axis (0 = x, 1 = y, 2 = z)."""
    comps = [a.copy() for a in g.split(v)]
    arr_axis = 2 - axis
    for c, a in enumerate(comps):
        if c == axis:          # the normal component: slots 0..n-1 are the faces
            sl = [slice(None)] * 3
            sl[arr_axis] = slice(0, a.shape[arr_axis] - 1)
            a[tuple(sl)] = np.roll(a[tuple(sl)], sh, axis=arr_axis)
        else:
            comps[c] = np.roll(a, sh, axis=arr_axis)
    return g.join(*comps)


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_periodic_operators_commute_with_periodic_shifts(axis):
    rng = np.random.default_rng(61)
    g = mac.Grid3(6, 4, 8, 1.0 / 6, periodic=True)
    v = rng.standard_normal(g.F) * g.interior_faces()
    u = rng.standard_normal(g.F) * g.interior_faces()
    rho = rng.random(g.C)
    sh = 2 if axis != 1 else 1
    rv = _roll(g, v, axis, sh)
    np.testing.assert_allclose(mac.adv(g, rv), _roll(g, mac.adv(g, v), axis, sh), atol=1e-12)
    np.testing.assert_allclose(mac.adv_jacobian_T_apply(g, rv, _roll(g, u, axis, sh)),
                               _roll(g, mac.adv_jacobian_T_apply(g, v, u), axis, sh), atol=1e-12)
    R = np.roll(rho.reshape(g.cell_shape()), sh, axis=2 - axis).ravel()
    AR = (mac.advection_matrix(g, rv) @ R).reshape(g.cell_shape())
    np.testing.assert_allclose(AR, np.roll((mac.advection_matrix(g, v) @ rho).reshape(g.cell_shape()), sh,
                                           axis=2 - axis), atol=1e-12)


def test_periodic_operators_equal_the_closed_ones_away_from_the_boundary():
    """Fields vanishing within three cells of every boundary plane: the wrap never
    reaches them, so div, grad, Adv, its transpose and QUICK agree with the
    closed-box operators."""
    rng = np.random.default_rng(62)
    n = 10
    gp = mac.Grid3(n, n, n, 1.0 / n, periodic=True)
    gc = mac.Grid3(n, n, n, 1.0 / n)
    sup = []
    for shape in gc.face_shapes():
        a = np.zeros(shape)
        a[3:-3, 3:-3, 3:-3] = 1.0
        sup.append(a)
    m = gc.join(*sup)
    v = rng.standard_normal(gc.F) * m
    u = rng.standard_normal(gc.F) * m
    rho = np.zeros(gc.cell_shape())
    rho[3:-3, 3:-3, 3:-3] = rng.random((n - 6,) * 3)
    rho = rho.ravel()
    np.testing.assert_allclose(mac.div(gp, v), mac.div(gc, v), atol=1e-12)
    np.testing.assert_allclose(mac.adv(gp, v), mac.adv(gc, v), atol=1e-12)
    np.testing.assert_allclose(mac.adv_jacobian_T_apply(gp, v, u), mac.adv_jacobian_T_apply(gc, v, u), atol=1e-12)
    np.testing.assert_allclose(mac.advection_matrix(gp, v) @ rho, mac.advection_matrix(gc, v) @ rho, atol=1e-12)
    p = rng.random(gc.C)
    interior = gc.interior_faces()
    np.testing.assert_allclose(mac.grad(gp, p) * interior, mac.grad(gc, p), atol=1e-12)


def test_periodic_projection_matches_the_fft_closed_form():
    rng = np.random.default_rng(63)
    g = mac.Grid3(8, 6, 4, 1.0 / 8, periodic=True)
    b = rng.standard_normal(g.C)
    b -= b.mean()
    B = np.fft.fftn(b.reshape(g.cell_shape()))
    lam = 0.0
    for axis, n in enumerate(g.cell_shape()):
        k = np.arange(n)
        shape = [1, 1, 1]
        shape[axis] = n
        lam = lam - (4 / g.h ** 2) * (np.sin(np.pi * k / n) ** 2).reshape(shape)
    lam = np.broadcast_to(lam, B.shape).copy()
    lam[0, 0, 0] = 1.0
    Pp = B / lam
    Pp[0, 0, 0] = 0.0
    np.testing.assert_allclose(projection.poisson_neumann(g, b), np.real(np.fft.ifftn(Pp)).ravel(), atol=1e-12)
    a = rng.standard_normal(g.F) * g.interior_faces()
    Qa = projection.project(g, a)
    assert np.max(np.abs(mac.div(g, Qa))) < 1e-10
    # a constant (harmonic) field is left alone: no walls remove it
    const = g.interior_faces() * 0.0
    cx, cy, cz = g.split(const)
    cx[:, :, :g.nx] = 1.0
    c = g.join(cx, cy, cz)
    np.testing.assert_allclose(projection.project(g, c), c, atol=1e-12)


def _problem3p(n=4, nz=4, N=3, **kw):
    rho0 = workloads.gaussian_ball3(n, n, nz, (0.5, 0.35, 0.5 * nz / n), 0.2)
    star = workloads.gaussian_ball3(n, n, nz, (0.5, 0.65, 0.45 * nz / n), 0.2)
    args = dict(r=1e-2, K=1.0, keyframes={N: (star, 1.0)}, metric_levels=1, nz=nz, periodic=True)
    args.update(kw)
    return kkt.Problem(n, n, N, 1.0 / N, rho0, **args)


def test_periodic_reduced_gradient_and_scgs_blocks():
    rng = np.random.default_rng(64)
    P = _problem3p()
    v = _solenoidal(P, rng, 0.4)
    _, Ks = kkt.forward_density(P, v)
    g = kkt.reduced_gradient(P, v)
    d = _solenoidal(P, rng, 1.0)
    eps = 1e-6
    fd = (kkt.objective(P, v + eps * d, Ks) - kkt.objective(P, v - eps * d, Ks)) / (2 * eps)
    an = float(np.sum(g * d))
    assert abs(fd - an) <= 1e-6 * max(abs(an), 1e-12), (fd, an)
    # the local blocks of the corner cell (its faces wrap) are FD columns of f
    P = _problem3p(lm_shift=0.0)
    x = _random_state(P, rng)
    x["u"][:] = 0.0
    gr = P.grid
    idx = (np.array([0]), np.array([0]), np.array([gr.nx - 1]))
    faces, active = scgs.cell_faces(gr, idx)
    assert np.all(active == 1.0)
    cell = gr.cell(*idx)[0]
    Dg, Lo, Up = scgs.assemble(P, gr, x, faces, active)
    A = scgs.dense_from_blocks(Dg[0], Lo[0], Up[0])
    z = np.zeros((P.N, gr.F))
    unk = []
    for i in range(P.N):
        unk += [("u", i, f) for f in faces[0]] + [("p", i, cell)]
        unk += [("v", i + 1, f) for f in faces[0]] + [("pbar", i + 1, cell)]
    f0 = kkt.nso_residual(P, gr, x, z)
    for col, (k, i, ix) in enumerate(unk):
        xp = kkt.copy_state(x)
        xp[k][i][ix] += eps
        fp = kkt.nso_residual(P, gr, xp, z)
        fdc = np.array([(fp[kk][ii][jx] - f0[kk][ii][jx]) / eps for kk, ii, jx in unk])
        np.testing.assert_allclose(A[:, col], fdc, atol=2e-4 * max(1.0, np.max(np.abs(fdc))))


def test_periodic_vcycles_converge_to_direct_solution():
    rng = np.random.default_rng(65)
    nx, nz, N = 8, 4, 2
    rho0 = workloads.gaussian_ball3(nx, nx, nz, (0.5, 0.35, 0.3), 0.2)
    P = kkt.Problem(nx, nx, N, 1.0 / N, rho0, r=1e-2, K=1.0, nz=nz, coarsest_n=2, periodic=True,
                    self_advection=False, keyframes={N: (rho0, 1.0)})
    assert [(g.nx, g.ny, g.nz) for g in stfas.hierarchy(P)] == [(8, 8, 4), (4, 4, 2)]
    z = np.array([projection.project(P.grid, w) for w in
                  rng.standard_normal((N, P.grid.F)) * P.grid.interior_faces()])
    ref = _linear_solution(P, z)
    x = kkt.zero_state(P)
    hist = [stfas.stfas_cycle(P, x, z) for _ in range(25)]
    for k in ("v", "u"):
        scale = max(np.max(np.abs(ref[k])), 1e-3 * np.max(np.abs(ref["u"])))
        np.testing.assert_allclose(x[k], ref[k], atol=1e-7 * scale)
    # pressures are defined up to a constant per step
    for k in ("pbar", "p"):
        d = x[k] - ref[k]
        d -= d.mean(axis=1, keepdims=True)
        assert np.max(np.abs(d)) < 1e-6 * max(1.0, np.max(np.abs(ref[k])))
    assert hist[-1] < 1e-8 * hist[0]
