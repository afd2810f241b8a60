"""Restriction, prolongation and the STFAS V-cycle, fp64.  Oracle -- test infrastructure only.

Sec. 4.2 / Alg. 2: a FAS V(2,2) cycle on a hierarchy coarsened in space only
(every timestep kept on every level), 10 smoothing sweeps on the coarsest
level, coarse right-hand side res^{2h} = f^{2h}(R x^h) + R(res^h - f^h(x^h)).

Readings:
* levels halve every axis while all are even and the halves are >= coarsest_n.
* R (Sec. 4.3 names trilinear interpolation): a coarse cell is the mean of
  its 2^d children; a coarse face the mean of the 2^(d-1) fine faces lying
  on it.
* P: (bi/tri)linear interpolation at the fine point -- cell fields (3/4, 1/4)
  per axis; face fields linear along the face normal (weights 1 or 1/2, 1/2)
  and (3/4, 1/4) across; indices beyond a wall clamp to the last coarse row.
* Alg. 2 subtracts P(R x^h) before evaluating f(x^h); here the fine residual
  is evaluated on the smoothed x^h and the correction is the usual
  x^h += P(x^{2h}_new - x^{2h}_old), which is what the subtract/add pair
  amounts to.
* the coarse target is z^{2h} = R z^h; the fine-level res is 0.
* coarse-grid correction guard (``P.cgc_guard``, default on): the correction
  is kept only if ||res - f(x + P e)||_2 <= ||res - f(x)||_2 on that level;
  otherwise x stays as the pre-smoothing left it.  Alg. 2 has no such test.
  Once the ADMM iterate carries strong flows (CFL of several cells per step),
  the unguarded cycle stalled at ||f||_inf ~ 1.7e2 on 32^2 x 16 (and
  diverged on 128^2 x 40) while the smoother alone kept reducing ||f||: the
  coarse correction undid the smoothing.  In the regime where the cycle
  contracts, the correction cuts the residual several-fold and is always kept,
  so the guard does not change the cycle there.
* time coarsening (``P.time_coarsen``, off by default: the paper coarsens in
  space only): while a level's N is even, the next level also halves N and
  doubles dt.  In time, point fields (v, pbar and their rows; the targets z)
  restrict by injection at the two ends and full weighting (1/4, 1/2, 1/4)
  inside, and prolong linearly; interval fields (u, p and their rows)
  restrict by the mean of the two sub-intervals and prolong piecewise
  constant.  Space and time transfers are applied one after the other.  The
  fine-level fixed point f = 0 does not depend on any of this.
"""
import dataclasses

import numpy as np

from . import kkt, mac, scgs


def _axes(g):
    return (g.nx, g.ny, g.nz) if g.dim == 3 else (g.nx, g.ny)


def hierarchy(P):
    grids = [P.grid]
    g = P.grid
    while all(n % 2 == 0 and n // 2 >= P.coarsest_n for n in _axes(g)):
        g = g.coarse()
        grids.append(g)
    return grids


def _pair_mean(X, axis):
    """Mean of the element pairs (2m, 2m+1) along ``axis``."""
    a = np.take(X, np.arange(0, X.shape[axis] - 1, 2), axis=axis)
    b = np.take(X, np.arange(1, X.shape[axis], 2), axis=axis)
    return 0.5 * (a + b)


def _even(X, axis):
    """Elements 0, 2, 4, ... along ``axis`` (fine faces on coarse faces)."""
    return np.take(X, np.arange(0, X.shape[axis], 2), axis=axis)


def restrict_cells(fine, x):
    if fine.dim == 3:
        X = x.reshape(fine.cell_shape())
        return _pair_mean(_pair_mean(_pair_mean(X, 0), 1), 2).ravel()
    X = x.reshape(fine.ny, fine.nx)
    return (0.25 * (X[0::2, 0::2] + X[0::2, 1::2] + X[1::2, 0::2] + X[1::2, 1::2])).ravel()


def restrict_faces(fine, v):
    if fine.dim == 3:
        # a coarse a-face: even fine a-faces along a, pair means across (axes k, j, i)
        vx, vy, vz = fine.split(v)
        cx = _even(_pair_mean(_pair_mean(vx, 0), 1), 2)
        cy = _even(_pair_mean(_pair_mean(vy, 0), 2), 1)
        cz = _even(_pair_mean(_pair_mean(vz, 1), 2), 0)
        return np.concatenate([cx.ravel(), cy.ravel(), cz.ravel()])
    vx, vy = fine.split(v)
    cx = 0.5 * (vx[0::2, 0::2] + vx[1::2, 0::2])      # (nyc, nxc+1)
    cy = 0.5 * (vy[0::2, 0::2] + vy[0::2, 1::2])      # (nyc+1, nxc)
    return np.concatenate([cx.ravel(), cy.ravel()])


def _interp_weights_cell(nf, nc):
    """Rows: fine index -> (coarse idx a, weight wa, coarse idx b, weight wb)."""
    k = np.arange(nf)
    a = k // 2
    b = np.where(k % 2 == 0, a - 1, a + 1)
    b = np.clip(b, 0, nc - 1)
    return a, b


def _interp_cells_axis(Xc, axis, nf, periodic=False):
    """(3/4, 1/4) interpolation of cell-centred data to nf fine cells along ``axis``
    (the far neighbour clamped at a wall, wrapped on a periodic axis)."""
    if periodic:
        k = np.arange(nf)
        a = k // 2
        b = np.where(k % 2 == 0, a - 1, a + 1) % Xc.shape[axis]
    else:
        a, b = _interp_weights_cell(nf, Xc.shape[axis])
    return 0.75 * np.take(Xc, a, axis=axis) + 0.25 * np.take(Xc, b, axis=axis)


def _interp_normal_axis(Xc, axis, nf_faces, periodic=False):
    """Linear interpolation of face data along the face normal (weights 1 or 1/2, 1/2);
    on a periodic axis the coarse face after the last is face 0."""
    if periodic:
        nc = Xc.shape[axis] - 1              # coarse faces 0..nc-1 (slot nc unused)
        k = np.arange(nf_faces)
        a = np.minimum(k // 2, nc - 1)
        b = (k // 2 + 1) % nc
        wb = np.where(k % 2 == 1, 0.5, 0.0)
        wa = np.where(k == nf_faces - 1, 0.0, 1.0 - wb)   # the unused fine slot stays zero
        wb = np.where(k == nf_faces - 1, 0.0, wb)
        shape = [1] * Xc.ndim
        shape[axis] = -1
        return np.take(Xc, a, axis=axis) * wa.reshape(shape) + np.take(Xc, b, axis=axis) * wb.reshape(shape)
    a, b, wa, wb = _interp_weights_normal(nf_faces, Xc.shape[axis])
    shape = [1] * Xc.ndim
    shape[axis] = -1
    return np.take(Xc, a, axis=axis) * wa.reshape(shape) + np.take(Xc, b, axis=axis) * wb.reshape(shape)


def prolong_cells(fine, coarse, xc):
    if fine.dim == 3:
        X = xc.reshape(coarse.cell_shape())
        for axis, nf in enumerate(fine.cell_shape()):
            X = _interp_cells_axis(X, axis, nf, fine.periodic)
        return X.ravel()
    Xc = xc.reshape(coarse.ny, coarse.nx)
    ay, by = _interp_weights_cell(fine.ny, coarse.ny)
    ax, bx = _interp_weights_cell(fine.nx, coarse.nx)
    rows = 0.75 * Xc[ay, :] + 0.25 * Xc[by, :]
    return (0.75 * rows[:, ax] + 0.25 * rows[:, bx]).ravel()


def _interp_weights_normal(nf_faces, nc_faces):
    """Fine face index k (0..nf) on the normal axis -> coarse faces (a, b), weights."""
    k = np.arange(nf_faces)
    a = k // 2
    b = np.minimum(a + 1, nc_faces - 1)
    wb = np.where(k % 2 == 1, 0.5, 0.0)
    return a, b, 1.0 - wb, wb


def prolong_faces(fine, coarse, vc):
    if fine.dim == 3:
        out = []
        for normal, X in zip((2, 1, 0), coarse.split(vc)):     # x-, y-, z-faces; axes (k, j, i)
            nfs = fine.face_shapes()[2 - normal]
            for axis in range(3):
                if axis == normal:
                    X = _interp_normal_axis(X, axis, nfs[axis], fine.periodic)
                else:
                    X = _interp_cells_axis(X, axis, nfs[axis], fine.periodic)
            out.append(X.ravel())
        return np.concatenate(out)
    cx, cy = coarse.split(vc)
    # x-faces: normal axis x (faces 0..nx), transverse axis y (cells)
    a, b, wa, wb = _interp_weights_normal(fine.nx + 1, coarse.nx + 1)
    ay, by = _interp_weights_cell(fine.ny, coarse.ny)
    t = 0.75 * cx[ay, :] + 0.25 * cx[by, :]
    fx = t[:, a] * wa + t[:, b] * wb
    # y-faces: normal axis y, transverse x
    a, b, wa, wb = _interp_weights_normal(fine.ny + 1, coarse.ny + 1)
    ax, bx = _interp_weights_cell(fine.nx, coarse.nx)
    t = 0.75 * cy[:, ax] + 0.25 * cy[:, bx]
    fy = t[a, :] * wa[:, None] + t[b, :] * wb[:, None]
    return np.concatenate([fx.ravel(), fy.ravel()])


def restrict_state(fine, x):
    return dict(v=np.array([restrict_faces(fine, a) for a in x["v"]]),
                pbar=np.array([restrict_cells(fine, a) for a in x["pbar"]]),
                u=np.array([restrict_faces(fine, a) for a in x["u"]]),
                p=np.array([restrict_cells(fine, a) for a in x["p"]]))


def prolong_state(fine, coarse, xc):
    return dict(v=np.array([prolong_faces(fine, coarse, a) for a in xc["v"]]),
                pbar=np.array([prolong_cells(fine, coarse, a) for a in xc["pbar"]]),
                u=np.array([prolong_faces(fine, coarse, a) for a in xc["u"]]),
                p=np.array([prolong_cells(fine, coarse, a) for a in xc["p"]]))


def restrict_faces_batch(fine, z):
    return np.array([restrict_faces(fine, a) for a in z])


def levels(P):
    """[(grid_l, P_l)] of the hierarchy: the grids of hierarchy(P); P_l = P with
    the level's N and dt (halved / doubled at every level while N is even when
    P.time_coarsen is set; the smoother's shift stays the finest level's)."""
    out = []
    Pl = P
    for l, g in enumerate(hierarchy(P)):
        if l > 0 and P.time_coarsen and Pl.N % 2 == 0:
            Pl = dataclasses.replace(Pl, N=Pl.N // 2, dt=2.0 * Pl.dt, lm_shift=P.lm_shift)
        out.append((g, Pl))
    return out


def restrict_time_points(a):
    """(N+1) point slabs -> (N/2+1): injection at 0 and N, full weighting inside.
    Also used for the N target slabs z_0..z_{N-1} (-> N/2), which have no end
    point to inject."""
    n = a.shape[0]
    if n % 2 == 1:                      # points 0..N
        nc = (n - 1) // 2 + 1
        out = np.empty((nc,) + a.shape[1:])
        out[0] = a[0]
        out[nc - 1] = a[n - 1]
    else:                               # targets 0..N-1
        nc = n // 2
        out = np.empty((nc,) + a.shape[1:])
        out[0] = a[0]
    for i in range(1, nc if n % 2 == 0 else nc - 1):
        out[i] = 0.25 * a[2 * i - 1] + 0.5 * a[2 * i] + 0.25 * a[2 * i + 1]
    return out


def restrict_time_intervals(a):
    """N interval slabs -> N/2: the mean of the two sub-intervals."""
    return 0.5 * (a[0::2] + a[1::2])


def prolong_time_points(ac):
    """(N/2+1) point slabs -> (N+1): linear interpolation."""
    nc = ac.shape[0]
    out = np.empty((2 * (nc - 1) + 1,) + ac.shape[1:])
    out[0::2] = ac
    out[1::2] = 0.5 * (ac[:-1] + ac[1:])
    return out


def prolong_time_intervals(ac):
    """N/2 interval slabs -> N: piecewise constant."""
    return np.repeat(ac, 2, axis=0)


def restrict_state_st(fine, x, in_time):
    xc = restrict_state(fine, x)
    if in_time:
        xc = dict(v=restrict_time_points(xc["v"]), pbar=restrict_time_points(xc["pbar"]),
                  u=restrict_time_intervals(xc["u"]), p=restrict_time_intervals(xc["p"]))
    return xc


def prolong_state_st(fine, coarse, xc, in_time):
    if in_time:
        xc = dict(v=prolong_time_points(xc["v"]), pbar=prolong_time_points(xc["pbar"]),
                  u=prolong_time_intervals(xc["u"]), p=prolong_time_intervals(xc["p"]))
    return prolong_state(fine, coarse, xc)


def restrict_targets(fine, z, in_time):
    zc = restrict_faces_batch(fine, z)
    return restrict_time_points(zc) if in_time else zc


def vcycle(P, grids, level, x, z, res):
    """One FAS V(pre, post) cycle on level ``level`` (in place on x).  ``grids``
    is hierarchy(P) (space only) or levels(P) (grid and per-level problem)."""
    g, Pl = grids[level] if isinstance(grids[level], tuple) else (grids[level], P)
    if level == len(grids) - 1:
        for _ in range(P.coarse_sweeps):
            scgs.sweep(Pl, g, x, z, res)
        return
    for _ in range(P.pre):
        scgs.sweep(Pl, g, x, z, res)
    f = kkt.nso_residual(Pl, g, x, z)
    rf = {k: res[k] - f[k] for k in f}
    gc, Pc = grids[level + 1] if isinstance(grids[level + 1], tuple) else (grids[level + 1], P)
    in_time = Pc.N != Pl.N
    xc = restrict_state_st(g, x, in_time)
    xc_old = kkt.copy_state(xc)
    zc = restrict_targets(g, z, in_time)
    fc = kkt.nso_residual(Pc, gc, xc, zc)
    rc = restrict_state_st(g, rf, in_time)
    resc = {k: fc[k] + rc[k] for k in fc}
    # rows dropped by the fixed v_0 stay zero
    resc["v"][0] = 0.0
    resc["pbar"][0] = 0.0
    vcycle(P, grids, level + 1, xc, zc, resc)
    corr = prolong_state_st(g, gc, kkt.state_sub(xc, xc_old), in_time)
    corr["v"][0] = 0.0      # v_0 is data, not an unknown
    corr["pbar"][0] = 0.0
    trial = {k: x[k] + corr[k] for k in x}
    if P.cgc_guard:
        # keep the coarse-grid correction only if it does not raise the
        # level's residual 2-norm; otherwise continue from the smoothed x
        ft = kkt.nso_residual(Pl, g, trial, z)
        before = sum(float(np.sum(a * a)) for a in rf.values())
        after = sum(float(np.sum((res[k] - ft[k]) ** 2)) for k in ft)
        if after <= before:
            for k in x:
                x[k] = trial[k]
    else:
        for k in x:
            x[k] = trial[k]
    for _ in range(P.post):
        scgs.sweep(Pl, g, x, z, res)


def normalise_pressures(x):
    """Remove each timestep's mean from pbar and p (their null space)."""
    x["pbar"] -= x["pbar"].mean(axis=1, keepdims=True)
    x["p"] -= x["p"].mean(axis=1, keepdims=True)


def stfas_cycle(P, x, z):
    """One top-level V-cycle for f(x) = 0 followed by pressure normalisation."""
    grids = levels(P)
    res = {k: np.zeros_like(a) for k, a in x.items()}
    vcycle(P, grids, 0, x, z, res)
    normalise_pressures(x)
    f = kkt.nso_residual(P, P.grid, x, z)
    return kkt.state_inf(f)
