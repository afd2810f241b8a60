"""Temporally augmented SCGS (Vanka) smoother, fp64.  Oracle -- test infrastructure only.

Sec. 4.3: one SCGS step solves, for one cell, the face unknowns v_i, u_i on its
faces together with the centre unknowns pbar_i, p_{i+1}, across all timesteps
at once; the local Jacobian is block tridiagonal in time (Eq. HESS) with
(2d+1)-blocks, and cells are 2^d-coloured so that one colour updates in
parallel.

Readings:
* block order B_u(0), B_v(1), B_u(1), ..., B_u(N-1), B_v(N) with
  B_v(i) = {v_i on the cell's faces, pbar_i}, B_u(i) = {u_i on the faces,
  p_{i+1}}; B_v(0) is absent because v_0 is fixed; wall faces are not unknowns.
* local matrix = the Eq. HESS restriction: diagonal blocks [[aI, g], [g^T, 0]]
  (a = K/r for i < N, 0 for i = N, plus the Levenberg-Marquardt shift gamma
  of Sec. 5, "a perturbation to the penalty coefficient K in the Hessian",
  default gamma = 1/dt^2 on every v block; it changes only the smoother, not
  the fixed point f = 0) and [[-I, g], [g^T, 0]]; couplings -I/dt
  between v_i and u_i, and I/dt + dAdv_loc(v_{i+1}) between u_i and v_{i+1}
  (and its transpose); g = d(grad p)/dp_c = (+1, -1, +1, -1)/h on the
  (left, right, bottom, top) faces, and (+1, -1)/h on the (back, front)
  z-faces in 3D.  The second-order term of Adv is dropped
  (Eq. HESS keeps only (K/r) I on the v diagonal).
* colours c = (i mod 2) + 2 (j mod 2) [+ 4 (k mod 2)] in increasing order; every cell of one
  colour is updated from the same state; under-relaxation x += omega * delta
  with omega = 0.8 by default (undamped sweeps diverge once the flow's CFL
  number passes 1; Vanka smoothers for Navier-Stokes are customarily damped).
* the block-tridiagonal system is solved by block Thomas elimination (the
  O(N) solve of Sec. 4.3), pinned against a dense solve.
"""
import numpy as np

from . import kkt, mac

def nfaces(grid):
    """2d faces per cell; a time block holds them and one pressure (2d + 1)."""
    return 2 * grid.dim


def cell_faces(grid, idx):
    """Local faces (left, right, bottom, top[, back, front]) of the cells with
    index arrays idx = (J, I) or (K, J, I), and their activity (1 = not a wall)."""
    if grid.dim == 3:
        K, J, I = idx
        if getattr(grid, "periodic", False):
            faces = np.stack([grid.xf(K, J, I), grid.xf(K, J, (I + 1) % grid.nx), grid.yf(K, J, I),
                              grid.yf(K, (J + 1) % grid.ny, I), grid.zf(K, J, I),
                              grid.zf((K + 1) % grid.nz, J, I)], -1)
            return faces, np.ones(faces.shape)
        faces = np.stack([grid.xf(K, J, I), grid.xf(K, J, I + 1), grid.yf(K, J, I),
                          grid.yf(K, J + 1, I), grid.zf(K, J, I), grid.zf(K + 1, J, I)], -1)
        active = np.stack([I > 0, I < grid.nx - 1, J > 0, J < grid.ny - 1,
                           K > 0, K < grid.nz - 1], -1).astype(float)
        return faces, active
    J, I = idx
    faces = np.stack([grid.xf(J, I), grid.xf(J, I + 1), grid.yf(J, I), grid.yf(J + 1, I)], -1)
    active = np.stack([I > 0, I < grid.nx - 1, J > 0, J < grid.ny - 1], -1).astype(float)
    return faces, active


_STATIC = {}


def _static_entries(grid, faces):
    """M[f, g] and T[f, g] of every bilinear term of Adv, for f, g among each
    cell's faces (fixed stencils)."""
    key = (grid.key(), faces.tobytes())
    if key not in _STATIC:
        nf = faces.shape[1]
        rows = np.repeat(faces[:, :, None], nf, axis=2).ravel()
        cols = np.repeat(faces[:, None, :], nf, axis=1).ravel()
        ent = []
        for M, T in mac.ops(grid)["terms"]:
            ent.append((np.asarray(M[rows, cols]).reshape(faces.shape[0], nf, nf),
                        np.asarray(T[rows, cols]).reshape(faces.shape[0], nf, nf)))
        _STATIC[key] = ent
    return _STATIC[key]


def local_adv_jacobian(grid, v, faces):
    """dAdv_f / dv_g for f, g among each cell's faces: (ncell, 2d, 2d).

    Entries of d Adv / d v = sum over terms of diag(T v) M + diag(M v) T at the
    local rows/columns."""
    out = 0.0
    for (M, T), (m, t) in zip(mac.ops(grid)["terms"], _static_entries(grid, faces)):
        out = out + (T @ v)[faces][:, :, None] * m + (M @ v)[faces][:, :, None] * t
    return out


def assemble(P, grid, x, faces, active):
    """Block-tridiagonal local Jacobians (Dg, Lo, Up), each (ncell, 2N, 2d+1, 2d+1)."""
    N, dt, h = P.N, P.dt, grid.h
    nc, nf = faces.shape
    NB = nf + 1
    nb = 2 * N
    Dg = np.zeros((nc, nb, NB, NB))
    Lo = np.zeros((nc, nb, NB, NB))
    Up = np.zeros((nc, nb, NB, NB))
    gl = active * np.tile([1.0, -1.0], nf // 2) / h             # (nc, 2d)
    Am = active[:, :, None] * active[:, None, :]                # active-pair mask
    eye = np.eye(nf)[None] * Am
    ina = np.eye(nf)[None] * (1.0 - active)[:, :, None]         # identity on walls
    for k in range(nb):
        if k % 2 == 0:      # B_u(i), i = k/2
            Dg[:, k, :nf, :nf] = -eye + ina
        else:               # B_v(i), i = (k+1)/2
            i = (k + 1) // 2
            a = (P.K / P.r if i < N else 0.0) + P.lm_shift
            Dg[:, k, :nf, :nf] = a * eye + ina
        Dg[:, k, :nf, nf] = gl
        Dg[:, k, nf, :nf] = gl
    for i in range(N):
        k = 2 * i
        sa = 1.0 if P.self_advection else 0.0
        M = (eye / dt + sa * local_adv_jacobian(grid, x["v"][i + 1], faces) * Am)
        Up[:, k, :nf, :nf] = M                        # J[B_u(i), B_v(i+1)]
        Lo[:, k + 1, :nf, :nf] = np.transpose(M, (0, 2, 1))   # J[B_v(i+1), B_u(i)]
        if i >= 1:
            Lo[:, k, :nf, :nf] = -eye / dt            # J[B_u(i), B_v(i)]
            Up[:, k - 1, :nf, :nf] = -eye / dt        # J[B_v(i), B_u(i)]
    return Dg, Lo, Up


def local_rhs(P, grid, r, faces, cells, active):
    """b = -(f - res) restricted to the local unknowns: (ncell, 2N, 2d+1)."""
    N = P.N
    nf = faces.shape[1]
    b = np.zeros((faces.shape[0], 2 * N, nf + 1))
    for i in range(N):
        b[:, 2 * i, :nf] = -r["u"][i][faces] * active
        b[:, 2 * i, nf] = -r["p"][i][cells]
        b[:, 2 * i + 1, :nf] = -r["v"][i + 1][faces] * active
        b[:, 2 * i + 1, nf] = -r["pbar"][i + 1][cells]
    return b


def block_thomas(Dg, Lo, Up, b):
    """Batched block-tridiagonal solve by block Gaussian elimination (no pivoting)."""
    nb = Dg.shape[1]
    Cp = np.zeros_like(Up)
    dp = np.zeros_like(b)
    M = Dg[:, 0]
    Cp[:, 0] = np.linalg.solve(M, Up[:, 0])
    dp[:, 0] = np.linalg.solve(M, b[:, 0][..., None])[..., 0]
    for k in range(1, nb):
        M = Dg[:, k] - Lo[:, k] @ Cp[:, k - 1]
        rhs = b[:, k] - (Lo[:, k] @ dp[:, k - 1][..., None])[..., 0]
        if k < nb - 1:
            Cp[:, k] = np.linalg.solve(M, Up[:, k])
        dp[:, k] = np.linalg.solve(M, rhs[..., None])[..., 0]
    x = np.zeros_like(b)
    x[:, nb - 1] = dp[:, nb - 1]
    for k in range(nb - 2, -1, -1):
        x[:, k] = dp[:, k] - (Cp[:, k] @ x[:, k + 1][..., None])[..., 0]
    return x


def dense_from_blocks(Dg, Lo, Up):
    """Assemble the dense (2N*(2d+1))^2 matrix of one cell's block-tridiagonal system."""
    nb = Dg.shape[0]
    NB = Dg.shape[1]
    A = np.zeros((nb * NB, nb * NB))
    for k in range(nb):
        A[k * NB:(k + 1) * NB, k * NB:(k + 1) * NB] = Dg[k]
        if k > 0:
            A[k * NB:(k + 1) * NB, (k - 1) * NB:k * NB] = Lo[k]
        if k < nb - 1:
            A[k * NB:(k + 1) * NB, (k + 1) * NB:(k + 2) * NB] = Up[k]
    return A


def colour_cells(grid, colour):
    """Index arrays (J, I) or (K, J, I) of the cells of one parity colour."""
    if grid.dim == 3:
        K, J, I = np.meshgrid(np.arange(grid.nz), np.arange(grid.ny), np.arange(grid.nx),
                              indexing="ij")
        sel = ((I % 2) + 2 * (J % 2) + 4 * (K % 2)) == colour
        return K[sel], J[sel], I[sel]
    J, I = np.meshgrid(np.arange(grid.ny), np.arange(grid.nx), indexing="ij")
    sel = ((I % 2) + 2 * (J % 2)) == colour
    return J[sel], I[sel]


def smooth_colour(P, grid, x, z, res, colour):
    """Update every cell of one colour from the same state (in place)."""
    idx = colour_cells(grid, colour)
    if idx[0].size == 0:
        return
    faces, active = cell_faces(grid, idx)
    nf = faces.shape[1]
    cells = grid.cell(*idx)
    f = kkt.nso_residual(P, grid, x, z)
    r = {k: f[k] - res[k] for k in f}
    Dg, Lo, Up = assemble(P, grid, x, faces, active)
    b = local_rhs(P, grid, r, faces, cells, active)
    d = P.omega * block_thomas(Dg, Lo, Up, b)
    N = P.N
    for i in range(N):
        x["u"][i][faces] += d[:, 2 * i, :nf] * active
        x["p"][i][cells] += d[:, 2 * i, nf]
        x["v"][i + 1][faces] += d[:, 2 * i + 1, :nf] * active
        x["pbar"][i + 1][cells] += d[:, 2 * i + 1, nf]


def sweep(P, grid, x, z, res):
    """One SCGS sweep: the 2^d colours in increasing order."""
    for colour in range(2 ** grid.dim):
        smooth_colour(P, grid, x, z, res, colour)
