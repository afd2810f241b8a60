"""Staggered (MAC) grid operators in 2D, fp64.  Oracle -- test infrastructure only.

The paper discretises velocity on cell faces and pressure / density at cell
centres (Sec. 3.1, "staggered grid").  Conventions fixed here:

* cells (j, i), 0 <= i < nx, 0 <= j < ny, centre ((i+1/2)h, (j+1/2)h);
  centre fields are arrays of shape (ny, nx), flattened with i fastest.
* x-faces (j, i), 0 <= i <= nx, at (ih, (j+1/2)h); y-faces (j, i),
  0 <= j <= ny, at ((i+1/2)h, jh).  A face vector holds all x-faces
  (ny*(nx+1), i fastest) followed by all y-faces ((ny+1)*nx, i fastest).
  Wall faces (i = 0, nx for x-faces; j = 0, ny for y-faces) are stored and
  are always zero: the box is closed (the paper's Neumann benchmarks, Table 1).
* nodes (j, i), 0 <= i <= nx, 0 <= j <= ny, at (ih, jh): vorticity lives here.

All operators are scipy.sparse matrices built from their stencil definitions.
"""
from functools import lru_cache

import numpy as np
import scipy.sparse as sp


class Grid:
    """Index bookkeeping for one nx-by-ny MAC grid with cell size h."""

    def __init__(self, nx, ny, h):
        self.nx, self.ny, self.h = int(nx), int(ny), float(h)
        self.C = self.nx * self.ny
        self.Fx = self.ny * (self.nx + 1)
        self.Fy = (self.ny + 1) * self.nx
        self.F = self.Fx + self.Fy
        self.Nn = (self.ny + 1) * (self.nx + 1)

    # flat indices -----------------------------------------------------------
    def cell(self, j, i):
        return j * self.nx + i

    def xf(self, j, i):
        return j * (self.nx + 1) + i

    def yf(self, j, i):
        return self.Fx + j * self.nx + i

    def node(self, j, i):
        return j * (self.nx + 1) + i

    # masks --------------------------------------------------------------------
    def interior_faces(self):
        m = np.zeros(self.F)
        mx = np.zeros((self.ny, self.nx + 1))
        mx[:, 1:self.nx] = 1.0
        my = np.zeros((self.ny + 1, self.nx))
        my[1:self.ny, :] = 1.0
        m[:self.Fx] = mx.ravel()
        m[self.Fx:] = my.ravel()
        return m

    def split(self, v):
        """View a face vector as (x-faces (ny, nx+1), y-faces (ny+1, nx))."""
        return (v[:self.Fx].reshape(self.ny, self.nx + 1),
                v[self.Fx:].reshape(self.ny + 1, self.nx))

    def join(self, vx, vy):
        return np.concatenate([np.asarray(vx).ravel(), np.asarray(vy).ravel()])

    def coarse(self):
        return Grid(self.nx // 2, self.ny // 2, 2.0 * self.h)

    def key(self):
        return (self.nx, self.ny, self.h)


def _sparse(entries, shape):
    """Assemble a CSR matrix from a list of (row_idx, col_idx, value) triples."""
    rows, cols, vals = [], [], []
    for r, c, v in entries:
        r = np.asarray(r)
        v = np.broadcast_to(np.asarray(v, dtype=float), r.shape).ravel()
        r = r.ravel()
        c = np.asarray(c).ravel()
        rows.append(r)
        cols.append(c)
        vals.append(v)
    if not rows:
        return sp.csr_matrix(shape)
    m = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=shape)
    return m.tocsr()


@lru_cache(maxsize=64)
def _ops(nx, ny, h):
    g = Grid(nx, ny, h)
    ih = 1.0 / h
    J, I = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")

    # divergence D (C x F): (div v)_c = sum_a (v_{a,c+} - v_{a,c-}) / h   (Eq. NSB)
    c = g.cell(J, I)
    D = _sparse([(c, g.xf(J, I + 1), ih), (c, g.xf(J, I), -ih),
                 (c, g.yf(J + 1, I), ih), (c, g.yf(J, I), -ih)], (g.C, g.F))

    # gradient G (F x C): (grad p)_f = (p_R - p_L) / h on interior faces, 0 on walls
    Jx, Ix = np.meshgrid(np.arange(ny), np.arange(1, nx), indexing="ij")
    Jy, Iy = np.meshgrid(np.arange(1, ny), np.arange(nx), indexing="ij")
    G = _sparse([(g.xf(Jx, Ix), g.cell(Jx, Ix), ih), (g.xf(Jx, Ix), g.cell(Jx, Ix - 1), -ih),
                 (g.yf(Jy, Iy), g.cell(Jy, Iy), ih), (g.yf(Jy, Iy), g.cell(Jy - 1, Iy), -ih)],
                (g.F, g.C))

    # vorticity W (nodes x F): omega = d v_y/dx - d v_x/dy at interior nodes,
    # zero at wall nodes (free slip).
    Jn, In = np.meshgrid(np.arange(1, ny), np.arange(1, nx), indexing="ij")
    nd = g.node(Jn, In)
    W = _sparse([(nd, g.yf(Jn, In), ih), (nd, g.yf(Jn, In - 1), -ih),
                 (nd, g.xf(Jn, In), -ih), (nd, g.xf(Jn - 1, In), ih)], (g.Nn, g.F))

    # node -> face average (F x nodes): the two nodes lying on each interior face
    Om = _sparse([(g.xf(Jx, Ix), g.node(Jx, Ix), 0.5), (g.xf(Jx, Ix), g.node(Jx + 1, Ix), 0.5),
                  (g.yf(Jy, Iy), g.node(Jy, Iy), 0.5), (g.yf(Jy, Iy), g.node(Jy, Iy + 1), 0.5)],
                 (g.F, g.Nn))

    # transverse average T (F x F): x-face <- the 4 surrounding y-faces and vice versa
    T = _sparse([(g.xf(Jx, Ix), g.yf(Jx, Ix - 1), 0.25), (g.xf(Jx, Ix), g.yf(Jx, Ix), 0.25),
                 (g.xf(Jx, Ix), g.yf(Jx + 1, Ix - 1), 0.25), (g.xf(Jx, Ix), g.yf(Jx + 1, Ix), 0.25),
                 (g.yf(Jy, Iy), g.xf(Jy - 1, Iy), 0.25), (g.yf(Jy, Iy), g.xf(Jy - 1, Iy + 1), 0.25),
                 (g.yf(Jy, Iy), g.xf(Jy, Iy), 0.25), (g.yf(Jy, Iy), g.xf(Jy, Iy + 1), 0.25)],
                (g.F, g.F))

    # sign of the Lamb vector component: (omega x v)_x = -omega v_y, (omega x v)_y = +omega v_x
    s = np.zeros(g.F)
    sx, sy = g.split(s)
    sx[:, 1:nx] = -1.0
    sy[1:ny, :] = 1.0
    s = g.join(sx, sy)
    OmW = (Om @ W).tocsr()
    return dict(grid=g, D=D, G=G, W=W, Om=Om, T=T, s=s, OmW=OmW, mask=g.interior_faces(),
                OmW_T=OmW.T.tocsr(), T_T=T.T.tocsr(), D_T=D.T.tocsr())


def ops(grid):
    return _ops(grid.nx, grid.ny, grid.h)


def div(grid, v):
    """Cell-centred divergence of a face field (Eq. NSB)."""
    return ops(grid)["D"] @ v


def grad(grid, p):
    """Face gradient of a centre field, zero on wall faces (Eq. NSA)."""
    return ops(grid)["G"] @ p


def vorticity(grid, v):
    """Node vorticity omega = dv_y/dx - dv_x/dy, zero at wall nodes."""
    return ops(grid)["W"] @ v


def adv(grid, v):
    """Self-advection Adv[v]: the Lamb vector (curl v) x v on faces (Sec. 3.1,
    Eq. NSA; "a discretization of the quadratic operator curl(.) x (.)").

    At an x-face: -omega_bar * vbar_y; at a y-face: +omega_bar * vbar_x, where
    omega_bar is the mean of the face's two nodes and vbar the mean of the four
    surrounding transverse faces.  Zero on wall faces.
    """
    o = ops(grid)
    return o["s"] * (o["OmW"] @ v) * (o["T"] @ v)


def adv_jacobian_factors(grid, v):
    """(a, b) with d Adv / d v = diag(a) OmW + diag(b) T (product rule of the
    bilinear form s * (OmW v) * (T v))."""
    o = ops(grid)
    return o["s"] * (o["T"] @ v), o["s"] * (o["OmW"] @ v)


def adv_jacobian(grid, v):
    """d Adv / d v at v as a sparse F x F matrix."""
    o = ops(grid)
    a, b = adv_jacobian_factors(grid, v)
    return (sp.diags(a) @ o["OmW"] + sp.diags(b) @ o["T"]).tocsr()


def adv_jacobian_T_apply(grid, v, u):
    """(d Adv / d v)^T u = OmW^T (a * u) + T^T (b * u)."""
    o = ops(grid)
    a, b = adv_jacobian_factors(grid, v)
    return o["OmW_T"] @ (a * u) + o["T_T"] @ (b * u)


# ---------------------------------------------------------------------------
# QUICK upwind passive advection (Sec. 3.1: "second order upwinding stencil",
# Leonard 1979), flux form.
# ---------------------------------------------------------------------------

def quick_face_matrix(grid, v):
    """Sparse F x C matrix mapping a centre field x to its QUICK face values.

    For an interior face between cells L (lower index) and R:
      v_f > 0: x_f = (6 x_L + 3 x_R - x_LL) / 8
      v_f < 0: x_f = (6 x_R + 3 x_L - x_RR) / 8
      v_f = 0: the mean of the two (the subgradient used for d/dv at v_f = 0).
    Cells beyond a wall clamp to the nearest interior cell.  Wall rows are zero.
    """
    g = grid
    nx, ny = g.nx, g.ny
    vx, vy = g.split(v)
    entries = []

    Jx, Ix = np.meshgrid(np.arange(ny), np.arange(1, nx), indexing="ij")
    wpos = np.where(vx[:, 1:nx] > 0, 1.0, np.where(vx[:, 1:nx] < 0, 0.0, 0.5))
    wneg = 1.0 - wpos
    f = g.xf(Jx, Ix)
    L, R = g.cell(Jx, Ix - 1), g.cell(Jx, Ix)
    LL, RR = g.cell(Jx, np.maximum(Ix - 2, 0)), g.cell(Jx, np.minimum(Ix + 1, nx - 1))
    entries += [(f, L, wpos * 6 / 8), (f, R, wpos * 3 / 8), (f, LL, -wpos / 8),
                (f, R, wneg * 6 / 8), (f, L, wneg * 3 / 8), (f, RR, -wneg / 8)]

    Jy, Iy = np.meshgrid(np.arange(1, ny), np.arange(nx), indexing="ij")
    wpos = np.where(vy[1:ny, :] > 0, 1.0, np.where(vy[1:ny, :] < 0, 0.0, 0.5))
    wneg = 1.0 - wpos
    f = g.yf(Jy, Iy)
    B, Tt = g.cell(Jy - 1, Iy), g.cell(Jy, Iy)
    BB, TT = g.cell(np.maximum(Jy - 2, 0), Iy), g.cell(np.minimum(Jy + 1, ny - 1), Iy)
    entries += [(f, B, wpos * 6 / 8), (f, Tt, wpos * 3 / 8), (f, BB, -wpos / 8),
                (f, Tt, wneg * 6 / 8), (f, B, wneg * 3 / 8), (f, TT, -wneg / 8)]
    return _sparse(entries, (g.F, g.C))


def advection_matrix(grid, v):
    """A(v): (A x)_c = -(1/h) sum_a (F_{c+1/2} - F_{c-1/2}), F_f = v_f x_f (QUICK)."""
    o = ops(grid)
    return (-(o["D"] @ sp.diags(v) @ quick_face_matrix(grid, v))).tocsr()


def advection_v_derivative_T(grid, v, x, mu):
    """B(x)^T mu where B(x) dv = d(A(v) x)/dv dv = -D (dv * x_face(v; x)).

    The upwind choice is frozen at v (A is piecewise linear in v); at v_f = 0 the
    face value is the mean of both one-sided choices.
    """
    o = ops(grid)
    xf = quick_face_matrix(grid, v) @ x
    return -(xf * (o["D"].T @ mu)) * o["mask"]


def advection_v_derivative(grid, v, x, dv):
    """B(x) dv (forward form, used by finite-difference and dot-product pins)."""
    o = ops(grid)
    xf = quick_face_matrix(grid, v) @ x
    return -(o["D"] @ (dv * o["mask"] * xf))
