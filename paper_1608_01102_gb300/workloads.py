"""Seeded synthetic inputs for the smoke-control workloads.

This module only draws and shapes input data (initial densities, keyframe
targets, random states for tests); it holds none of the method's arithmetic
and is shared by the CUDA path's tests/bench and the fp64 oracle's callers.

Recipes (the paper's keyframe shapes -- letters, bunny, armadillo, mocap --
are not available, so these stand in for them):

* ``gaussian_ball``: exp(-|x - c|^2 / (2 sigma^2)) at cell centres of the unit
  square.
* ``disc_bar_union``: the max of 3-5 shapes, each with probability 1/2 a disc
  (centre U[0.2, 0.8]^2, radius U[0.05, 0.12]) or an axis-aligned bar (width
  U[0.04, 0.08], length U[0.2, 0.5], orientation a coin flip); the indicator is
  Gaussian-blurred (sigma in cells, clamped edges) and scaled to a given mass.
* ``ellipsoid_union`` (3D): the max of 2-4 axis-aligned ellipsoids (centre
  U[0.25, 0.75]^3, semi-axes U[0.05, 0.2]), blurred (sigma in cells) and
  scaled to a given mass.
* 3D arrays are (nz, ny, nx) with i fastest; face vectors hold the x-, y- and
  z-faces in that order, each (k, j, i) with i fastest.
"""
import math

import numpy as np


def cell_centres(nx, ny):
    h = 1.0 / nx
    x = (np.arange(nx) + 0.5) * h
    y = (np.arange(ny) + 0.5) * h
    return np.meshgrid(x, y)          # arrays (ny, nx)


def gaussian_ball(nx, ny, centre, sigma):
    X, Y = cell_centres(nx, ny)
    return np.exp(-((X - centre[0]) ** 2 + (Y - centre[1]) ** 2) / (2.0 * sigma * sigma)).ravel()


def _blur_axis(a, sigma, axis):
    R = int(math.ceil(3.0 * sigma))
    t = np.arange(-R, R + 1)
    w = np.exp(-t * t / (2.0 * sigma * sigma))
    w /= w.sum()
    n = a.shape[axis]
    out = np.zeros_like(a)
    for k, wk in zip(t, w):
        idx = np.clip(np.arange(n) + k, 0, n - 1)
        out += wk * np.take(a, idx, axis=axis)
    return out


def disc_bar_union(nx, ny, seed, mass, blur_cells=1.5, count=None):
    rng = np.random.default_rng(seed)
    X, Y = cell_centres(nx, ny)
    m = np.zeros((ny, nx))
    k = int(rng.integers(3, 6)) if count is None else count
    for _ in range(k):
        if rng.random() < 0.5:
            c = rng.uniform(0.2, 0.8, 2)
            r = rng.uniform(0.05, 0.12)
            m = np.maximum(m, ((X - c[0]) ** 2 + (Y - c[1]) ** 2 <= r * r).astype(float))
        else:
            c = rng.uniform(0.2, 0.8, 2)
            w = rng.uniform(0.04, 0.08)
            L = rng.uniform(0.2, 0.5)
            if rng.random() < 0.5:
                hw, hh = L / 2, w / 2
            else:
                hw, hh = w / 2, L / 2
            m = np.maximum(m, ((np.abs(X - c[0]) <= hw) & (np.abs(Y - c[1]) <= hh)).astype(float))
    m = _blur_axis(_blur_axis(m, blur_cells, 0), blur_cells, 1)
    s = m.sum()
    return (m * (mass / s)).ravel() if s > 0 else m.ravel()


def face_count(nx, ny):
    return ny * (nx + 1) + (ny + 1) * nx


def interior_face_mask(nx, ny):
    mx = np.zeros((ny, nx + 1))
    mx[:, 1:nx] = 1.0
    my = np.zeros((ny + 1, nx))
    my[1:ny, :] = 1.0
    return np.concatenate([mx.ravel(), my.ravel()])


def random_faces(rng, nx, ny, count, scale=1.0):
    """Random face fields, zero on wall faces: (count, F)."""
    m = interior_face_mask(nx, ny)
    return rng.standard_normal((count, face_count(nx, ny))) * m * scale


def swirl_velocity(nx, ny, amplitude, centre=(0.5, 0.5), width=0.25):
    """A smooth vortex-like face field (zero on walls), for non-trivial states."""
    h = 1.0 / nx
    xs = np.arange(nx + 1) * h
    ys = (np.arange(ny) + 0.5) * h
    X, Y = np.meshgrid(xs, ys)
    g = np.exp(-((X - centre[0]) ** 2 + (Y - centre[1]) ** 2) / (2 * width ** 2))
    vx = -(Y - centre[1]) * g * amplitude
    vx[:, 0] = 0.0
    vx[:, nx] = 0.0
    xs = (np.arange(nx) + 0.5) * h
    ys = np.arange(ny + 1) * h
    X, Y = np.meshgrid(xs, ys)
    g = np.exp(-((X - centre[0]) ** 2 + (Y - centre[1]) ** 2) / (2 * width ** 2))
    vy = (X - centre[0]) * g * amplitude
    vy[0, :] = 0.0
    vy[ny, :] = 0.0
    return np.concatenate([vx.ravel(), vy.ravel()])


def cell_centres3(nx, ny, nz):
    h = 1.0 / nx
    z, y, x = ((np.arange(n) + 0.5) * h for n in (nz, ny, nx))
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    return X, Y, Z                    # arrays (nz, ny, nx)


def gaussian_ball3(nx, ny, nz, centre, sigma):
    X, Y, Z = cell_centres3(nx, ny, nz)
    d2 = (X - centre[0]) ** 2 + (Y - centre[1]) ** 2 + (Z - centre[2]) ** 2
    return np.exp(-d2 / (2.0 * sigma * sigma)).ravel()


def ellipsoid_union(nx, ny, nz, seed, mass, blur_cells=1.0, count=None):
    rng = np.random.default_rng(seed)
    X, Y, Z = cell_centres3(nx, ny, nz)
    m = np.zeros((nz, ny, nx))
    k = int(rng.integers(2, 5)) if count is None else count
    for _ in range(k):
        c = rng.uniform(0.25, 0.75, 3)
        a = rng.uniform(0.05, 0.2, 3)
        q = ((X - c[0]) / a[0]) ** 2 + ((Y - c[1]) / a[1]) ** 2 + ((Z - c[2]) / a[2]) ** 2
        m = np.maximum(m, (q <= 1.0).astype(float))
    for axis in range(3):
        m = _blur_axis(m, blur_cells, axis)
    s = m.sum()
    return (m * (mass / s)).ravel() if s > 0 else m.ravel()


def face_count3(nx, ny, nz):
    return nz * ny * (nx + 1) + nz * (ny + 1) * nx + (nz + 1) * ny * nx


def interior_face_mask3(nx, ny, nz, periodic=False):
    """1 on the face unknowns: interior faces of the closed box, or every face
    slot but the unused slot n of each axis on the periodic grid."""
    lo = 0 if periodic else 1
    mx = np.zeros((nz, ny, nx + 1))
    mx[:, :, lo:nx] = 1.0
    my = np.zeros((nz, ny + 1, nx))
    my[:, lo:ny, :] = 1.0
    mz = np.zeros((nz + 1, ny, nx))
    mz[lo:nz] = 1.0
    return np.concatenate([mx.ravel(), my.ravel(), mz.ravel()])


def random_faces3(rng, nx, ny, nz, count, scale=1.0, periodic=False):
    """Random 3D face fields, zero on wall faces (on the unused slots if periodic): (count, F)."""
    m = interior_face_mask3(nx, ny, nz, periodic)
    return rng.standard_normal((count, face_count3(nx, ny, nz))) * m * scale


def swirl_velocity3(nx, ny, nz, amplitude, centre=(0.5, 0.5, 0.5), width=0.25):
    """A smooth face field rotating about the z axis with a Gaussian envelope
    and a weak vertical component (zero on walls), for non-trivial 3D states."""
    h = 1.0 / nx
    def pos(axis):
        shp = [(nz, ny, nx + 1), (nz, ny + 1, nx), (nz + 1, ny, nx)][axis]
        ax = [np.arange(n) * h if a == 2 - axis else (np.arange(n) + 0.5) * h
              for a, n in enumerate(shp)]
        Z, Y, X = np.meshgrid(*ax, indexing="ij")
        return X, Y, Z
    out = []
    for axis in range(3):
        X, Y, Z = pos(axis)
        g = np.exp(-((X - centre[0]) ** 2 + (Y - centre[1]) ** 2 + (Z - centre[2]) ** 2)
                   / (2 * width ** 2)) * amplitude
        f = [-(Y - centre[1]) * g, (X - centre[0]) * g, 0.25 * (X - centre[0]) * g][axis]
        out.append(f.ravel())
    return np.concatenate(out) * interior_face_mask3(nx, ny, nz)


def _fftn(a):
    try:
        import scipy.fft
        return scipy.fft.fftn(a, workers=-1)
    except ImportError:
        return np.fft.fftn(a)


def _ifftn(a):
    try:
        import scipy.fft
        return scipy.fft.ifftn(a, workers=-1)
    except ImportError:
        return np.fft.ifftn(a)


def gaussian_random_faces3(nx, ny, nz, count, seed, corr_cells=8.0, amplitude=0.1):
    """Seeded smooth random 3D face fields (count, F): per slab and face axis,
    white noise filtered by a Gaussian of standard deviation corr_cells cells
    (FFT, periodic), the whole set scaled to max |u| = amplitude, zero on wall
    faces.  (Gradient parts are left in: every implicit step projects them
    out.)"""
    rng = np.random.default_rng(seed)
    shapes = [(nz, ny, nx + 1), (nz, ny + 1, nx), (nz + 1, ny, nx)]
    out = np.zeros((count, face_count3(nx, ny, nz)))
    for c in range(count):
        parts = []
        for shp in shapes:
            w = rng.standard_normal(shp)
            k = [np.fft.fftfreq(n) for n in shp]
            K2 = sum(np.meshgrid(*[q * q for q in k], indexing="ij"))
            filt = np.exp(-2.0 * (np.pi * corr_cells) ** 2 * K2)
            parts.append(np.real(_ifftn(_fftn(w) * filt)).ravel())
        out[c] = np.concatenate(parts)
    out *= interior_face_mask3(nx, ny, nz)[None]
    return out * (amplitude / np.max(np.abs(out)))


def config_autograd(n=128, N=48, seed=5005):
    """The differentiable-simulation workload: n^3 cells, N steps, dt = 1/N;
    initial density a Gaussian ball (sigma 0.1) at (0.5, 0.35, 0.5); forces a
    seeded smooth random field (correlation length 8 cells, max |u| = 0.1);
    target rho* a seeded union of ellipsoids blurred by one cell, mass-matched."""
    rho0 = gaussian_ball3(n, n, n, (0.5, 0.35, 0.5), 0.1)
    rng = np.random.default_rng(seed)
    star = ellipsoid_union(n, n, n, int(rng.integers(0, 2**31 - 1)), rho0.sum(), 1.0)
    u = gaussian_random_faces3(n, n, n, N, int(rng.integers(0, 2**31 - 1)), 8.0, 0.1)
    return dict(nx=n, ny=n, nz=n, N=N, dt=1.0 / N, rho0=rho0, star=star, u=u)


def config_small(n=32, N=16):
    """2D, n^2 cells, N steps, dt = 1/N: ball (sigma 0.08) at (0.5, 0.3) to the
    same ball at (0.5, 0.7) at t = T, zero initial velocity, r = 1e-3."""
    rho0 = gaussian_ball(n, n, (0.5, 0.3), 0.08)
    star = gaussian_ball(n, n, (0.5, 0.7), 0.08)
    return dict(nx=n, ny=n, N=N, dt=1.0 / N, rho0=rho0, keyframes={N: (star, 1.0)}, r=1e-3)


def config_letters(n=128, N=40, seed=2002):
    """2D, 128^2 cells, 40 steps: ball (sigma 0.08) at (0.5, 0.25) to a seeded,
    blurred (1.5 cells), mass-matched disc/bar union at t = T, r = 1e-3."""
    rho0 = gaussian_ball(n, n, (0.5, 0.25), 0.08)
    star = disc_bar_union(n, n, seed, rho0.sum(), 1.5)
    return dict(nx=n, ny=n, N=N, dt=1.0 / N, rho0=rho0, keyframes={N: (star, 1.0)}, r=1e-3)


def config_3d(n=64, N=60, seed=3003):
    """3D, n^3 cells, N steps, dt = 1/N: ball (sigma 0.1) at (0.5, 0.2, 0.5);
    keyframes at steps N/2 and N (30 and 60 for N = 60), each a seeded union of
    2-4 ellipsoids blurred by 1 cell and scaled to the initial mass; r = 1e-3."""
    rho0 = gaussian_ball3(n, n, n, (0.5, 0.2, 0.5), 0.1)
    rng = np.random.default_rng(seed)
    kf = {}
    for step in (N // 2, N):
        kf[step] = (ellipsoid_union(n, n, n, int(rng.integers(0, 2**31 - 1)), rho0.sum(), 1.0), 1.0)
    return dict(nx=n, ny=n, nz=n, N=N, dt=1.0 / N, rho0=rho0, keyframes=kf, r=1e-3)


def config_serving(count=256, seed=4004, rate=4.0):
    """A stream of 2D control requests: Poisson arrivals at ``rate`` per second
    (exponential gaps), n uniform over {32, 48, 64, 96, 128}, N uniform in
    [16, 48] (dt = 1/N), m uniform over {1, 2, 3} keyframes at steps
    round(j N / m), each a seeded blurred (1.5 cells) disc/bar union with the
    initial mass; the initial density is the ball of config_letters; r = 1e-3.
    Returns a list of dicts (the config_letters keys plus ``arrival`` in s)."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for k in range(count):
        t += rng.exponential(1.0 / rate)
        n = int(rng.choice([32, 48, 64, 96, 128]))
        N = int(rng.integers(16, 49))
        m = int(rng.integers(1, 4))
        rho0 = gaussian_ball(n, n, (0.5, 0.25), 0.08)
        kf = {}
        for j in range(1, m + 1):
            step = int(round(j * N / m))
            kf[step] = (disc_bar_union(n, n, int(rng.integers(0, 2**31 - 1)), rho0.sum(), 1.5), 1.0)
        out.append(dict(nx=n, ny=n, N=N, dt=1.0 / N, rho0=rho0, keyframes=kf, r=1e-3, arrival=t))
    return out
