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
  (left, right, bottom, top) faces.  The second-order term of Adv is dropped
  (Eq. HESS keeps only (K/r) I on the v diagonal).
* colours c = (i mod 2) + 2 (j mod 2) in increasing order; every cell of one
  colour is updated from the same state; under-relaxation x += omega * delta
  with omega = 0.8 by default (undamped sweeps diverge once the flow's CFL
  number passes 1; Vanka smoothers for Navier-Stokes are customarily damped).
* the block-tridiagonal system is solved by block Thomas elimination (the
  O(N) solve of Sec. 4.3), pinned against a dense solve.
"""
import numpy as np

from . import kkt, mac

NB = 5  # 2d + 1 unknowns per block in 2D


def cell_faces(grid, J, I):
    """Local faces (left, right, bottom, top) of cells (J, I) and their activity."""
    faces = np.stack([grid.xf(J, I), grid.xf(J, I + 1), grid.yf(J, I), grid.yf(J + 1, I)], -1)
    active = np.stack([I > 0, I < grid.nx - 1, J > 0, J < grid.ny - 1], -1).astype(float)
    return faces, active


_STATIC = {}


def _static_entries(grid, faces):
    """OmW[f, g] and T[f, g] for f, g among each cell's faces (fixed stencils)."""
    key = (grid.key(), faces.tobytes())
    if key not in _STATIC:
        o = mac.ops(grid)
        rows = np.repeat(faces[:, :, None], 4, axis=2).ravel()
        cols = np.repeat(faces[:, None, :], 4, axis=1).ravel()
        om = np.asarray(o["OmW"][rows, cols]).reshape(faces.shape[0], 4, 4)
        tt = np.asarray(o["T"][rows, cols]).reshape(faces.shape[0], 4, 4)
        _STATIC[key] = (om, tt)
    return _STATIC[key]


def local_adv_jacobian(grid, v, faces):
    """dAdv_f / dv_g for f, g among each cell's four faces: (ncell, 4, 4).

    Entries of d Adv / d v = diag(a) OmW + diag(b) T at the local rows/columns."""
    om, tt = _static_entries(grid, faces)
    a, b = mac.adv_jacobian_factors(grid, v)
    return a[faces][:, :, None] * om + b[faces][:, :, None] * tt


def assemble(P, grid, x, faces, active):
    """Block-tridiagonal local Jacobians (Dg, Lo, Up), each (ncell, 2N, 5, 5)."""
    N, dt, h = P.N, P.dt, grid.h
    nc = faces.shape[0]
    nb = 2 * N
    Dg = np.zeros((nc, nb, NB, NB))
    Lo = np.zeros((nc, nb, NB, NB))
    Up = np.zeros((nc, nb, NB, NB))
    gl = active * np.array([1.0, -1.0, 1.0, -1.0]) / h          # (nc, 4)
    Am = active[:, :, None] * active[:, None, :]                # active-pair mask
    eye = np.eye(4)[None] * Am
    ina = np.eye(4)[None] * (1.0 - active)[:, :, None]          # identity on walls
    for k in range(nb):
        if k % 2 == 0:      # B_u(i), i = k/2
            Dg[:, k, :4, :4] = -eye + ina
        else:               # B_v(i), i = (k+1)/2
            i = (k + 1) // 2
            a = (P.K / P.r if i < N else 0.0) + P.lm_shift
            Dg[:, k, :4, :4] = a * eye + ina
        Dg[:, k, :4, 4] = gl
        Dg[:, k, 4, :4] = gl
    for i in range(N):
        k = 2 * i
        sa = 1.0 if P.self_advection else 0.0
        M = (eye / dt + sa * local_adv_jacobian(grid, x["v"][i + 1], faces) * Am)
        Up[:, k, :4, :4] = M                          # J[B_u(i), B_v(i+1)]
        Lo[:, k + 1, :4, :4] = np.transpose(M, (0, 2, 1))   # J[B_v(i+1), B_u(i)]
        if i >= 1:
            Lo[:, k, :4, :4] = -eye / dt              # J[B_u(i), B_v(i)]
            Up[:, k - 1, :4, :4] = -eye / dt          # J[B_v(i), B_u(i)]
    return Dg, Lo, Up


def local_rhs(P, grid, r, faces, cells, active):
    """b = -(f - res) restricted to the local unknowns: (ncell, 2N, 5)."""
    N = P.N
    b = np.zeros((faces.shape[0], 2 * N, NB))
    for i in range(N):
        b[:, 2 * i, :4] = -r["u"][i][faces] * active
        b[:, 2 * i, 4] = -r["p"][i][cells]
        b[:, 2 * i + 1, :4] = -r["v"][i + 1][faces] * active
        b[:, 2 * i + 1, 4] = -r["pbar"][i + 1][cells]
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
    """Assemble the dense (2N*5)^2 matrix of one cell's block-tridiagonal system."""
    nb = Dg.shape[0]
    A = np.zeros((nb * NB, nb * NB))
    for k in range(nb):
        A[k * NB:(k + 1) * NB, k * NB:(k + 1) * NB] = Dg[k]
        if k > 0:
            A[k * NB:(k + 1) * NB, (k - 1) * NB:k * NB] = Lo[k]
        if k < nb - 1:
            A[k * NB:(k + 1) * NB, (k + 1) * NB:(k + 2) * NB] = Up[k]
    return A


def colour_cells(grid, colour):
    J, I = np.meshgrid(np.arange(grid.ny), np.arange(grid.nx), indexing="ij")
    sel = ((I % 2) + 2 * (J % 2)) == colour
    return J[sel], I[sel]


def smooth_colour(P, grid, x, z, res, colour):
    """Update every cell of one colour from the same state (in place)."""
    J, I = colour_cells(grid, colour)
    if J.size == 0:
        return
    faces, active = cell_faces(grid, J, I)
    cells = grid.cell(J, I)
    f = kkt.nso_residual(P, grid, x, z)
    r = {k: f[k] - res[k] for k in f}
    Dg, Lo, Up = assemble(P, grid, x, faces, active)
    b = local_rhs(P, grid, r, faces, cells, active)
    d = P.omega * block_thomas(Dg, Lo, Up, b)
    N = P.N
    for i in range(N):
        x["u"][i][faces] += d[:, 2 * i, :4] * active
        x["p"][i][cells] += d[:, 2 * i, 4]
        x["v"][i + 1][faces] += d[:, 2 * i + 1, :4] * active
        x["pbar"][i + 1][cells] += d[:, 2 * i + 1, 4]


def sweep(P, grid, x, z, res):
    """One SCGS sweep: the 2^d colours in increasing order."""
    for colour in range(4):
        smooth_colour(P, grid, x, z, res, colour)
