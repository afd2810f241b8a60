"""Staggered (MAC) grid operators in 2D and 3D, fp64.  Oracle -- test infrastructure only.

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

3D (Grid3) is the same with a third axis: cells (k, j, i), i fastest; x-, y-
and z-faces in that order, each block (k, j, i) with i fastest; vorticity
components on edges (omega_x on x-edges at ((i+1/2)h, jh, kh), omega_y on
y-edges at (ih, (j+1/2)h, kh), omega_z on z-edges at (ih, jh, (k+1/2)h)),
zero on edges lying in a wall.

All operators are scipy.sparse matrices built from their stencil definitions.
"""
from functools import lru_cache

import numpy as np
import scipy.sparse as sp


class Grid:
    """Index bookkeeping for one nx-by-ny MAC grid with cell size h."""

    dim = 2
    nz = 1

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

    def cell_shape(self):
        return (self.ny, self.nx)


class Grid3:
    """Index bookkeeping for one nx-by-ny-by-nz MAC grid with cell size h.

    periodic=True: every axis wraps (no walls).  The face layout keeps n + 1
    slots per axis; slot n is not a face (it stays zero) and face 0 lies
    between cells n-1 and 0.  Edges and neighbour indices wrap likewise."""

    dim = 3

    def __init__(self, nx, ny, nz, h, periodic=False):
        self.nx, self.ny, self.nz, self.h = int(nx), int(ny), int(nz), float(h)
        self.periodic = bool(periodic)
        self.C = self.nx * self.ny * self.nz
        self.Fx = self.nz * self.ny * (self.nx + 1)
        self.Fy = self.nz * (self.ny + 1) * self.nx
        self.Fz = (self.nz + 1) * self.ny * self.nx
        self.F = self.Fx + self.Fy + self.Fz
        self.Ex = (self.nz + 1) * (self.ny + 1) * self.nx
        self.Ey = (self.nz + 1) * self.ny * (self.nx + 1)
        self.Ez = self.nz * (self.ny + 1) * (self.nx + 1)

    # flat indices -----------------------------------------------------------
    def cell(self, k, j, i):
        return (k * self.ny + j) * self.nx + i

    def xf(self, k, j, i):
        return (k * self.ny + j) * (self.nx + 1) + i

    def yf(self, k, j, i):
        return self.Fx + (k * (self.ny + 1) + j) * self.nx + i

    def zf(self, k, j, i):
        return self.Fx + self.Fy + (k * self.ny + j) * self.nx + i

    def xe(self, k, j, i):
        return (k * (self.ny + 1) + j) * self.nx + i

    def ye(self, k, j, i):
        return (k * self.ny + j) * (self.nx + 1) + i

    def ze(self, k, j, i):
        return (k * (self.ny + 1) + j) * (self.nx + 1) + i

    def face_shapes(self):
        return ((self.nz, self.ny, self.nx + 1), (self.nz, self.ny + 1, self.nx),
                (self.nz + 1, self.ny, self.nx))

    def interior_faces(self):
        lo = 0 if self.periodic else 1
        mx = np.zeros(self.face_shapes()[0])
        mx[:, :, lo:self.nx] = 1.0
        my = np.zeros(self.face_shapes()[1])
        my[:, lo:self.ny, :] = 1.0
        mz = np.zeros(self.face_shapes()[2])
        mz[lo:self.nz] = 1.0
        return self.join(mx, my, mz)

    def split(self, v):
        """View a face vector as (x-, y-, z-faces), each shaped (k, j, i)."""
        a, b = self.Fx, self.Fx + self.Fy
        sx, sy, sz = self.face_shapes()
        return v[:a].reshape(sx), v[a:b].reshape(sy), v[b:].reshape(sz)

    def join(self, vx, vy, vz):
        return np.concatenate([np.asarray(vx).ravel(), np.asarray(vy).ravel(),
                               np.asarray(vz).ravel()])

    def coarse(self):
        return Grid3(self.nx // 2, self.ny // 2, self.nz // 2, 2.0 * self.h, self.periodic)

    def key(self):
        return (self.nx, self.ny, self.nz, self.h, self.periodic)

    def cell_shape(self):
        return (self.nz, self.ny, self.nx)


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
    M = (sp.diags(s) @ OmW).tocsr()
    return dict(grid=g, D=D, G=G, W=W, Om=Om, T=T, s=s, OmW=OmW, mask=g.interior_faces(),
                OmW_T=OmW.T.tocsr(), T_T=T.T.tocsr(), D_T=D.T.tocsr(),
                terms=[(M, T.tocsr())], terms_T=[(M.T.tocsr(), T.T.tocsr())])


@lru_cache(maxsize=16)
def _ops3(nx, ny, nz, h):
    g = Grid3(nx, ny, nz, h)
    ih = 1.0 / h
    ar = np.arange

    def mesh(kr, jr, ir):
        return np.meshgrid(kr, jr, ir, indexing="ij")

    # divergence D (C x F) and gradient G (F x C), as in 2D with a third axis
    K, J, I = mesh(ar(nz), ar(ny), ar(nx))
    c = g.cell(K, J, I)
    D = _sparse([(c, g.xf(K, J, I + 1), ih), (c, g.xf(K, J, I), -ih),
                 (c, g.yf(K, J + 1, I), ih), (c, g.yf(K, J, I), -ih),
                 (c, g.zf(K + 1, J, I), ih), (c, g.zf(K, J, I), -ih)], (g.C, g.F))
    Kx, Jx, Ix = mesh(ar(nz), ar(ny), ar(1, nx))          # interior x-faces
    Ky, Jy, Iy = mesh(ar(nz), ar(1, ny), ar(nx))          # interior y-faces
    Kz, Jz, Iz = mesh(ar(1, nz), ar(ny), ar(nx))          # interior z-faces
    G = _sparse([(g.xf(Kx, Jx, Ix), g.cell(Kx, Jx, Ix), ih), (g.xf(Kx, Jx, Ix), g.cell(Kx, Jx, Ix - 1), -ih),
                 (g.yf(Ky, Jy, Iy), g.cell(Ky, Jy, Iy), ih), (g.yf(Ky, Jy, Iy), g.cell(Ky, Jy - 1, Iy), -ih),
                 (g.zf(Kz, Jz, Iz), g.cell(Kz, Jz, Iz), ih), (g.zf(Kz, Jz, Iz), g.cell(Kz - 1, Jz, Iz), -ih)],
                (g.F, g.C))

    # curl on interior edges (zero on edges lying in a wall):
    #   omega_x = d v_z/dy - d v_y/dz,  omega_y = d v_x/dz - d v_z/dx,  omega_z = d v_y/dx - d v_x/dy
    Ke, Je, Ie = mesh(ar(1, nz), ar(1, ny), ar(nx))
    e = g.xe(Ke, Je, Ie)
    Wx = _sparse([(e, g.zf(Ke, Je, Ie), ih), (e, g.zf(Ke, Je - 1, Ie), -ih),
                  (e, g.yf(Ke, Je, Ie), -ih), (e, g.yf(Ke - 1, Je, Ie), ih)], (g.Ex, g.F))
    Ke, Je, Ie = mesh(ar(1, nz), ar(ny), ar(1, nx))
    e = g.ye(Ke, Je, Ie)
    Wy = _sparse([(e, g.xf(Ke, Je, Ie), ih), (e, g.xf(Ke - 1, Je, Ie), -ih),
                  (e, g.zf(Ke, Je, Ie), -ih), (e, g.zf(Ke, Je, Ie - 1), ih)], (g.Ey, g.F))
    Ke, Je, Ie = mesh(ar(nz), ar(1, ny), ar(1, nx))
    e = g.ze(Ke, Je, Ie)
    Wz = _sparse([(e, g.yf(Ke, Je, Ie), ih), (e, g.yf(Ke, Je, Ie - 1), -ih),
                  (e, g.xf(Ke, Je, Ie), -ih), (e, g.xf(Ke, Je - 1, Ie), ih)], (g.Ez, g.F))

    # edge -> face means (the two edges of a component lying on an interior face)
    # and transverse face means (the four faces of a component around a face)
    fx, fy, fz = g.xf(Kx, Jx, Ix), g.yf(Ky, Jy, Iy), g.zf(Kz, Jz, Iz)
    Oy_x = _sparse([(fx, g.ye(Kx, Jx, Ix), .5), (fx, g.ye(Kx + 1, Jx, Ix), .5)], (g.F, g.Ey))
    Oz_x = _sparse([(fx, g.ze(Kx, Jx, Ix), .5), (fx, g.ze(Kx, Jx + 1, Ix), .5)], (g.F, g.Ez))
    Oz_y = _sparse([(fy, g.ze(Ky, Jy, Iy), .5), (fy, g.ze(Ky, Jy, Iy + 1), .5)], (g.F, g.Ez))
    Ox_y = _sparse([(fy, g.xe(Ky, Jy, Iy), .5), (fy, g.xe(Ky + 1, Jy, Iy), .5)], (g.F, g.Ex))
    Ox_z = _sparse([(fz, g.xe(Kz, Jz, Iz), .5), (fz, g.xe(Kz, Jz + 1, Iz), .5)], (g.F, g.Ex))
    Oy_z = _sparse([(fz, g.ye(Kz, Jz, Iz), .5), (fz, g.ye(Kz, Jz, Iz + 1), .5)], (g.F, g.Ey))
    q = 0.25
    Tz_x = _sparse([(fx, g.zf(Kx, Jx, Ix - 1), q), (fx, g.zf(Kx, Jx, Ix), q),
                    (fx, g.zf(Kx + 1, Jx, Ix - 1), q), (fx, g.zf(Kx + 1, Jx, Ix), q)], (g.F, g.F))
    Ty_x = _sparse([(fx, g.yf(Kx, Jx, Ix - 1), q), (fx, g.yf(Kx, Jx, Ix), q),
                    (fx, g.yf(Kx, Jx + 1, Ix - 1), q), (fx, g.yf(Kx, Jx + 1, Ix), q)], (g.F, g.F))
    Tx_y = _sparse([(fy, g.xf(Ky, Jy - 1, Iy), q), (fy, g.xf(Ky, Jy - 1, Iy + 1), q),
                    (fy, g.xf(Ky, Jy, Iy), q), (fy, g.xf(Ky, Jy, Iy + 1), q)], (g.F, g.F))
    Tz_y = _sparse([(fy, g.zf(Ky, Jy - 1, Iy), q), (fy, g.zf(Ky, Jy, Iy), q),
                    (fy, g.zf(Ky + 1, Jy - 1, Iy), q), (fy, g.zf(Ky + 1, Jy, Iy), q)], (g.F, g.F))
    Ty_z = _sparse([(fz, g.yf(Kz - 1, Jz, Iz), q), (fz, g.yf(Kz - 1, Jz + 1, Iz), q),
                    (fz, g.yf(Kz, Jz, Iz), q), (fz, g.yf(Kz, Jz + 1, Iz), q)], (g.F, g.F))
    Tx_z = _sparse([(fz, g.xf(Kz - 1, Jz, Iz), q), (fz, g.xf(Kz - 1, Jz, Iz + 1), q),
                    (fz, g.xf(Kz, Jz, Iz), q), (fz, g.xf(Kz, Jz, Iz + 1), q)], (g.F, g.F))

    # Lamb vector (omega x v)_a = omega_{a+1} v_{a+2} - omega_{a+2} v_{a+1} (cyclic):
    # term 1 = (+omega_{a+1}) * vbar_{a+2}, term 2 = (-omega_{a+2}) * vbar_{a+1}
    M1 = (Oy_x @ Wy + Oz_y @ Wz + Ox_z @ Wx).tocsr()
    T1 = (Tz_x + Tx_y + Ty_z).tocsr()
    M2 = (-(Oz_x @ Wz + Ox_y @ Wx + Oy_z @ Wy)).tocsr()
    T2 = (Ty_x + Tz_y + Tx_z).tocsr()
    terms = [(M1, T1), (M2, T2)]
    return dict(grid=g, D=D, G=G, Wx=Wx, Wy=Wy, Wz=Wz, mask=g.interior_faces(), D_T=D.T.tocsr(),
                terms=terms, terms_T=[(a.T.tocsr(), b.T.tocsr()) for a, b in terms])


@lru_cache(maxsize=16)
def _ops3p(nx, ny, nz, h):
    """The operators of _ops3 on the triply periodic grid: the same stencils
    with every neighbour index taken modulo the axis length; all faces with
    normal index < n are faces, all edges interior."""
    g = Grid3(nx, ny, nz, h, periodic=True)
    ih = 1.0 / h
    ar = np.arange

    def mesh(kr, jr, ir):
        return np.meshgrid(kr, jr, ir, indexing="ij")

    wx, wy, wz = (lambda a: a % nx), (lambda a: a % ny), (lambda a: a % nz)
    K, J, I = mesh(ar(nz), ar(ny), ar(nx))
    c = g.cell(K, J, I)
    D = _sparse([(c, g.xf(K, J, wx(I + 1)), ih), (c, g.xf(K, J, I), -ih),
                 (c, g.yf(K, wy(J + 1), I), ih), (c, g.yf(K, J, I), -ih),
                 (c, g.zf(wz(K + 1), J, I), ih), (c, g.zf(K, J, I), -ih)], (g.C, g.F))
    fx, fy, fz = g.xf(K, J, I), g.yf(K, J, I), g.zf(K, J, I)     # every face, indexed by (k, j, i)
    G = _sparse([(fx, g.cell(K, J, I), ih), (fx, g.cell(K, J, wx(I - 1)), -ih),
                 (fy, g.cell(K, J, I), ih), (fy, g.cell(K, wy(J - 1), I), -ih),
                 (fz, g.cell(K, J, I), ih), (fz, g.cell(wz(K - 1), J, I), -ih)], (g.F, g.C))
    ex, ey, ez = g.xe(K, J, I), g.ye(K, J, I), g.ze(K, J, I)      # every edge, indexed by (k, j, i)
    Wx = _sparse([(ex, g.zf(K, J, I), ih), (ex, g.zf(K, wy(J - 1), I), -ih),
                  (ex, g.yf(K, J, I), -ih), (ex, g.yf(wz(K - 1), J, I), ih)], (g.Ex, g.F))
    Wy = _sparse([(ey, g.xf(K, J, I), ih), (ey, g.xf(wz(K - 1), J, I), -ih),
                  (ey, g.zf(K, J, I), -ih), (ey, g.zf(K, J, wx(I - 1)), ih)], (g.Ey, g.F))
    Wz = _sparse([(ez, g.yf(K, J, I), ih), (ez, g.yf(K, J, wx(I - 1)), -ih),
                  (ez, g.xf(K, J, I), -ih), (ez, g.xf(K, wy(J - 1), I), ih)], (g.Ez, g.F))
    Oy_x = _sparse([(fx, g.ye(K, J, I), .5), (fx, g.ye(wz(K + 1), J, I), .5)], (g.F, g.Ey))
    Oz_x = _sparse([(fx, g.ze(K, J, I), .5), (fx, g.ze(K, wy(J + 1), I), .5)], (g.F, g.Ez))
    Oz_y = _sparse([(fy, g.ze(K, J, I), .5), (fy, g.ze(K, J, wx(I + 1)), .5)], (g.F, g.Ez))
    Ox_y = _sparse([(fy, g.xe(K, J, I), .5), (fy, g.xe(wz(K + 1), J, I), .5)], (g.F, g.Ex))
    Ox_z = _sparse([(fz, g.xe(K, J, I), .5), (fz, g.xe(K, wy(J + 1), I), .5)], (g.F, g.Ex))
    Oy_z = _sparse([(fz, g.ye(K, J, I), .5), (fz, g.ye(K, J, wx(I + 1)), .5)], (g.F, g.Ey))
    q = 0.25
    im, jm, km = wx(I - 1), wy(J - 1), wz(K - 1)
    ip, jp, kp = wx(I + 1), wy(J + 1), wz(K + 1)
    Tz_x = _sparse([(fx, g.zf(K, J, im), q), (fx, g.zf(K, J, I), q),
                    (fx, g.zf(kp, J, im), q), (fx, g.zf(kp, J, I), q)], (g.F, g.F))
    Ty_x = _sparse([(fx, g.yf(K, J, im), q), (fx, g.yf(K, J, I), q),
                    (fx, g.yf(K, jp, im), q), (fx, g.yf(K, jp, I), q)], (g.F, g.F))
    Tx_y = _sparse([(fy, g.xf(K, jm, I), q), (fy, g.xf(K, jm, ip), q),
                    (fy, g.xf(K, J, I), q), (fy, g.xf(K, J, ip), q)], (g.F, g.F))
    Tz_y = _sparse([(fy, g.zf(K, jm, I), q), (fy, g.zf(K, J, I), q),
                    (fy, g.zf(kp, jm, I), q), (fy, g.zf(kp, J, I), q)], (g.F, g.F))
    Ty_z = _sparse([(fz, g.yf(km, J, I), q), (fz, g.yf(km, jp, I), q),
                    (fz, g.yf(K, J, I), q), (fz, g.yf(K, jp, I), q)], (g.F, g.F))
    Tx_z = _sparse([(fz, g.xf(km, J, I), q), (fz, g.xf(km, J, ip), q),
                    (fz, g.xf(K, J, I), q), (fz, g.xf(K, J, ip), q)], (g.F, g.F))
    M1 = (Oy_x @ Wy + Oz_y @ Wz + Ox_z @ Wx).tocsr()
    T1 = (Tz_x + Tx_y + Ty_z).tocsr()
    M2 = (-(Oz_x @ Wz + Ox_y @ Wx + Oy_z @ Wy)).tocsr()
    T2 = (Ty_x + Tz_y + Tx_z).tocsr()
    terms = [(M1, T1), (M2, T2)]
    return dict(grid=g, D=D, G=G, Wx=Wx, Wy=Wy, Wz=Wz, mask=g.interior_faces(), D_T=D.T.tocsr(),
                terms=terms, terms_T=[(a.T.tocsr(), b.T.tocsr()) for a, b in terms])


def ops(grid):
    if grid.dim == 3 and getattr(grid, "periodic", False):
        return _ops3p(grid.nx, grid.ny, grid.nz, grid.h)
    if grid.dim == 3:
        return _ops3(grid.nx, grid.ny, grid.nz, grid.h)
    return _ops(grid.nx, grid.ny, grid.h)


def div(grid, v):
    """Cell-centred divergence of a face field (Eq. NSB)."""
    return ops(grid)["D"] @ v


def grad(grid, p):
    """Face gradient of a centre field, zero on wall faces (Eq. NSA)."""
    return ops(grid)["G"] @ p


def vorticity(grid, v):
    """Node vorticity omega = dv_y/dx - dv_x/dy, zero at wall nodes (2D); in 3D
    the tuple (omega_x, omega_y, omega_z) on the edges."""
    o = ops(grid)
    if grid.dim == 3:
        return o["Wx"] @ v, o["Wy"] @ v, o["Wz"] @ v
    return o["W"] @ v


def adv(grid, v):
    """Self-advection Adv[v]: the Lamb vector (curl v) x v on faces (Sec. 3.1,
    Eq. NSA; "a discretization of the quadratic operator curl(.) x (.)").

    2D: at an x-face -omega_bar * vbar_y, at a y-face +omega_bar * vbar_x, with
    omega_bar the mean of the face's two nodes and vbar the mean of the four
    surrounding transverse faces.  3D: (omega x v)_a = omega_{a+1} v_{a+2} -
    omega_{a+2} v_{a+1}, each omega component the mean of the two edges of
    that component on the face, each v component the mean of its four faces
    around the face.  Zero on wall faces.  Written as a sum of bilinear terms
    (M v) * (T v) (one in 2D, two in 3D).
    """
    out = np.zeros(grid.F)
    for M, T in ops(grid)["terms"]:
        out += (M @ v) * (T @ v)
    return out


def adv_jacobian(grid, v):
    """d Adv / d v at v as a sparse F x F matrix (product rule on every term)."""
    J = sp.csr_matrix((grid.F, grid.F))
    for M, T in ops(grid)["terms"]:
        J = J + sp.diags(T @ v) @ M + sp.diags(M @ v) @ T
    return J.tocsr()


def adv_jacobian_T_apply(grid, v, u):
    """(d Adv / d v)^T u = sum over terms of M^T ((T v) u) + T^T ((M v) u)."""
    o = ops(grid)
    out = np.zeros(grid.F)
    for (M, T), (MT, TT) in zip(o["terms"], o["terms_T"]):
        out += MT @ ((T @ v) * u) + TT @ ((M @ v) * u)
    return out


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
    if grid.dim == 3:
        return _quick_face_matrix3(grid, v)
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


def _quick_weights(vn):
    """(upwind-from-lower, upwind-from-upper) weights of a face from its normal velocity."""
    wpos = np.where(vn > 0, 1.0, np.where(vn < 0, 0.0, 0.5))
    return wpos, 1.0 - wpos


def _quick_face_matrix3p(g, v):
    """QUICK face values on the periodic grid: faces 0..n-1 of every axis,
    lower cell p-1 and the far cells taken modulo n."""
    nx, ny, nz = g.nx, g.ny, g.nz
    vx, vy, vz = g.split(v)
    K, J, I = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    entries = []
    for axis, (vn, n) in enumerate(((vx[:, :, :nx], nx), (vy[:, :ny, :], ny), (vz[:nz], nz))):
        wp, wn = _quick_weights(vn)
        crd = [I, J, K][axis]

        def cell(p):
            c = [K, J, I]
            c[2 - axis] = p % n
            return g.cell(*c)

        f = [g.xf, g.yf, g.zf][axis](K, J, I)
        L, R, LL, RR = cell(crd - 1), cell(crd), cell(crd - 2), cell(crd + 1)
        entries += [(f, L, wp * 6 / 8), (f, R, wp * 3 / 8), (f, LL, -wp / 8),
                    (f, R, wn * 6 / 8), (f, L, wn * 3 / 8), (f, RR, -wn / 8)]
    return _sparse(entries, (g.F, g.C))


def _quick_face_matrix3(g, v):
    if g.periodic:
        return _quick_face_matrix3p(g, v)
    nx, ny, nz = g.nx, g.ny, g.nz
    vx, vy, vz = g.split(v)
    ar = np.arange
    entries = []
    K, J, I = np.meshgrid(ar(nz), ar(ny), ar(1, nx), indexing="ij")
    wp, wn = _quick_weights(vx[:, :, 1:nx])
    f = g.xf(K, J, I)
    L, R = g.cell(K, J, I - 1), g.cell(K, J, I)
    LL, RR = g.cell(K, J, np.maximum(I - 2, 0)), g.cell(K, J, np.minimum(I + 1, nx - 1))
    entries += [(f, L, wp * 6 / 8), (f, R, wp * 3 / 8), (f, LL, -wp / 8),
                (f, R, wn * 6 / 8), (f, L, wn * 3 / 8), (f, RR, -wn / 8)]
    K, J, I = np.meshgrid(ar(nz), ar(1, ny), ar(nx), indexing="ij")
    wp, wn = _quick_weights(vy[:, 1:ny, :])
    f = g.yf(K, J, I)
    L, R = g.cell(K, J - 1, I), g.cell(K, J, I)
    LL, RR = g.cell(K, np.maximum(J - 2, 0), I), g.cell(K, np.minimum(J + 1, ny - 1), I)
    entries += [(f, L, wp * 6 / 8), (f, R, wp * 3 / 8), (f, LL, -wp / 8),
                (f, R, wn * 6 / 8), (f, L, wn * 3 / 8), (f, RR, -wn / 8)]
    K, J, I = np.meshgrid(ar(1, nz), ar(ny), ar(nx), indexing="ij")
    wp, wn = _quick_weights(vz[1:nz])
    f = g.zf(K, J, I)
    L, R = g.cell(K - 1, J, I), g.cell(K, J, I)
    LL, RR = g.cell(np.maximum(K - 2, 0), J, I), g.cell(np.minimum(K + 1, nz - 1), J, I)
    entries += [(f, L, wp * 6 / 8), (f, R, wp * 3 / 8), (f, LL, -wp / 8),
                (f, R, wn * 6 / 8), (f, L, wn * 3 / 8), (f, RR, -wn / 8)]
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
