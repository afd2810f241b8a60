"""Keyframe metric C_i = c_i sum_l G_l^T G_l, fp64.  Oracle -- test infrastructure only.

Sec. 4.1: C_i is a sum of Gaussian filters whose standard deviation doubles
from one to the next.  Readings (the paper gives no sigma_0, truncation or
count): sigma_l = sigma_0 * 2^l cells, l = 0..L-1, taps truncated at
ceil(3 sigma_l), weights normalised to sum 1, clamp-to-edge boundary, separable
in x and y (and z on a 3D grid).  L = 0 gives C_i = c_i I (the plain
objective of Eq. opt).
"""
import math

import numpy as np


def default_levels(n):
    """L = floor(log2(n / 2)) filters for an n-cell axis (32 -> 4, 128 -> 6)."""
    return int(math.floor(math.log2(n / 2))) if n >= 2 else 0


def gaussian_taps(sigma):
    R = int(math.ceil(3.0 * sigma))
    t = np.arange(-R, R + 1, dtype=float)
    w = np.exp(-t * t / (2.0 * sigma * sigma))
    return w / w.sum()


def blur_matrix_1d(n, sigma, periodic=False):
    """n x n matrix of one normalised, truncated Gaussian blur, clamp-to-edge
    (or wrapping around on a periodic axis)."""
    w = gaussian_taps(sigma)
    R = (len(w) - 1) // 2
    M = np.zeros((n, n))
    for a in range(n):
        for t in range(-R, R + 1):
            b = (a + t) % n if periodic else min(max(a + t, 0), n - 1)
            M[a, b] += w[t + R]
    return M


def apply_metric(nx, ny, x, levels, sigma0=1.0, c=1.0, nz=0, periodic=False):
    """C x = c sum_l G_l^T G_l x for a centre field x (flattened, i fastest);
    nz > 0 makes it a 3D field of shape (nz, ny, nx); periodic: the filters wrap."""
    shape = (nz, ny, nx) if nz else (ny, nx)
    X = x.reshape(shape)
    if levels == 0:
        return c * x.copy()
    out = np.zeros_like(X)
    for l in range(levels):
        s = sigma0 * 2.0 ** l
        mats = [blur_matrix_1d(n, s, periodic) for n in shape]     # one per axis
        GX = X
        for ax, M in enumerate(mats):                    # G_l x
            GX = np.moveaxis(np.tensordot(M, GX, axes=([1], [ax])), 0, ax)
        for ax, M in enumerate(mats):                    # G_l^T (G_l x)
            GX = np.moveaxis(np.tensordot(M.T, GX, axes=([1], [ax])), 0, ax)
        out += GX
    return c * out.ravel()


def metric_matrix(nx, ny, levels, sigma0=1.0, c=1.0, nz=0):
    """Dense C (for small-grid pins only)."""
    n = nx * ny * max(nz, 1)
    M = np.zeros((n, n))
    for k in range(n):
        e = np.zeros(n)
        e[k] = 1.0
        M[:, k] = apply_metric(nx, ny, e, levels, sigma0, c, nz)
    return M
