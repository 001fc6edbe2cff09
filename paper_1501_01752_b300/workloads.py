"""Seeded synthetic inputs shared by the CUDA path, the tests and the bench.

This module holds geometry, incident points and random numbers only: none of
the method's arithmetic (no Fourier images, no operator, no solver, no pole
fit).  It is the single place both the CUDA path and the CPU oracle take
their inputs from.

Units: the vacuum wavelength is 1, so k0 = 2 pi; periods are in wavelengths.
A shape is (kind, center[3], size[3], eps) with kind SPHERE (size[0] = radius),
BOX (full side lengths) or ELLIPSOID (semi-axes); centres are in the cell
[0, Lambda_x) x [0, Lambda_y) x [0, Lambda_z).
"""
from __future__ import annotations

import math

import numpy as np

SPHERE, BOX, ELLIPSOID = 0, 1, 2
K0 = 2.0 * math.pi


def sphere_lattice(period=0.3, radius_frac=0.3, eps=4.0):
    """Simple-cubic lattice of spheres at the cell centre in a host of eps 1
    (the 7-harmonic FP64 single solve: eps 4, R = 0.3 Lambda, Lambda = 0.3)."""
    L = float(period)
    return dict(periods=(L, L, L), eps_host=1.0,
                shapes=[(SPHERE, (L / 2, L / 2, L / 2), (radius_frac * L, 0.0, 0.0), eps)])


def woodpile(period=0.35, eps=11.9, width_frac=0.25):
    """Two-layer woodpile: the layer z in [0, L/2) holds one rod along x
    (width 0.25 L in y, centred at y = 0), the layer z in [L/2, L) one rod
    along y (width 0.25 L in x, centred at x = 0).  Fill factor 0.25."""
    L = float(period)
    w = width_frac * L
    return dict(periods=(L, L, L), eps_host=1.0,
                shapes=[(BOX, (L / 2, 0.0, L / 4), (L, w, L / 2), eps),
                        (BOX, (0.0, L / 2, 3 * L / 4), (w, L, L / 2), eps)])


def ellipsoid_lattice(period=0.3, eps=6.0, semi=(0.4, 0.3, 0.2)):
    """Lattice of triaxial ellipsoids (semi-axes 0.4/0.3/0.2 Lambda), host 1."""
    L = float(period)
    return dict(periods=(L, L, L), eps_host=1.0,
                shapes=[(ELLIPSOID, (L / 2, L / 2, L / 2), tuple(s * L for s in semi), eps)])


def cavity_lattice(period=0.3, host_n=1.5, cube_side_frac=None, sphere_radius=None):
    """Air cavities (cubes of side cube_side_frac*L, or spheres of radius
    sphere_radius in wavelengths) in a host of index host_n."""
    L = float(period)
    c = (L / 2, L / 2, L / 2)
    if cube_side_frac is not None:
        s = cube_side_frac * L
        shapes = [(BOX, c, (s, s, s), 1.0)]
    else:
        shapes = [(SPHERE, c, (float(sphere_radius), 0.0, 0.0), 1.0)]
    return dict(periods=(L, L, L), eps_host=host_n**2, shapes=shapes)


def layered_stack(period=0.3, d1_frac=0.5, eps1=1.0, eps2=4.0, axis=2):
    """1D stack along `axis`: a layer of eps2 and thickness (1-d1_frac) L in a
    host of eps1 (box spanning the other two periods)."""
    L = float(period)
    size = [L, L, L]
    size[axis] = (1.0 - d1_frac) * L
    center = [L / 2, L / 2, L / 2]
    return dict(periods=(L, L, L), eps_host=eps1, shapes=[(BOX, tuple(center), tuple(size), eps2)])


def random_binary_voxels(M=64, seed=1501, sigma=2.0, fill=0.3, eps=(1.0, 6.0), mirror=False):
    """Seeded Gaussian-smoothed random binary field on an M^3 grid: iid
    N(0, 1) (numpy PCG64), periodic Gaussian smoothing of sigma voxels,
    threshold at the (1 - fill) quantile.  mirror=True averages the smoothed
    field over the mirrors x, y, z -> -x, -y, -z about the cell centre before
    thresholding, so the cell has orthorhombic symmetry and principal axes
    along x, y, z.  Returns eps[v_z, v_y, v_x]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    g = rng.standard_normal((M, M, M))
    f = np.fft.fftfreq(M)
    fz, fy, fx = np.meshgrid(f, f, f, indexing="ij")
    kernel = np.exp(-2.0 * (math.pi * sigma) ** 2 * (fx**2 + fy**2 + fz**2))
    s = np.fft.ifftn(np.fft.fftn(g) * kernel).real
    if mirror:
        s = s + s[::-1, :, :]
        s = s + s[:, ::-1, :]
        s = s + s[:, :, ::-1]
    thr = np.quantile(s, 1.0 - fill)
    return np.where(s > thr, eps[1], eps[0]).astype(np.float64)


def gyroid_voxels(M=128, level=0.5, eps=(1.0, 12.0)):
    """Gyroid solid g > level sampled at the M^3 voxel centres,
    g = sin X cos Y + sin Y cos Z + sin Z cos X, X = 2 pi (v + 1/2) / M."""
    t = 2.0 * math.pi * (np.arange(M) + 0.5) / M
    Z, Y, X = np.meshgrid(t, t, t, indexing="ij")
    g = np.sin(X) * np.cos(Y) + np.sin(Y) * np.cos(Z) + np.sin(Z) * np.cos(X)
    return np.where(g > level, eps[1], eps[0]).astype(np.float64)


def random_shapes(seed, period=(0.3, 0.33, 0.36), n=3):
    """A seeded asymmetric structure (non-overlapping boxes, a sphere and an
    ellipsoid at off-centre positions) for operator parity tests."""
    rng = np.random.Generator(np.random.PCG64(seed))
    Lx, Ly, Lz = period
    shapes = []
    for i in range(n):
        zc = (i + 0.5) * Lz / n
        kind = (BOX, SPHERE, ELLIPSOID)[i % 3]
        cx, cy = rng.uniform(0, Lx), rng.uniform(0, Ly)
        r = 0.4 * min(Lx, Ly, Lz / n) * rng.uniform(0.5, 1.0)
        if kind == BOX:
            size = (rng.uniform(0.2, 0.8) * Lx, rng.uniform(0.2, 0.8) * Ly, 0.8 * Lz / n)
        elif kind == SPHERE:
            size = (r, 0.0, 0.0)
        else:
            size = (r, 0.8 * r, 0.6 * r)
        shapes.append((kind, (cx, cy, zc), size, float(rng.uniform(2.0, 12.0))))
    return dict(periods=tuple(period), eps_host=float(rng.uniform(1.0, 2.0)), shapes=shapes)


def random_field(n_harm, seed, batch=None):
    """Seeded complex normal field of shape ([batch,] 3, N_z, N_y, N_x)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    shape = (3, n_harm[2], n_harm[1], n_harm[0])
    if batch is not None:
        shape = (batch,) + shape
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def unit(v):
    v = np.asarray(v, float)
    return v / np.linalg.norm(v)


def point(kappa, kdir=(0.0, 0.0, 1.0), pol=(1.0, 0.0, 0.0), k0=K0):
    """One incident point: k0, direction, |k_inc| = kappa, polarisation a."""
    return dict(k0=float(k0), kdir=tuple(unit(kdir)), kappa=float(kappa),
                pol=tuple(complex(p) for p in pol))


def kappa_grid(k0, n_centre, rel=0.15, M=16):
    """M equidistant kappa over k0 n_centre [1 - rel, 1 + rel]."""
    return k0 * n_centre * (1.0 + rel * np.linspace(-1.0, 1.0, M))


def woodpile_batch(B=32, k0=K0):
    """B single-solve points for the 31-harmonic woodpile: kappa spread over
    [0.70, 0.90] k0 (below the basis light cone, away from the mode pole),
    alternating x and y polarisation, normal incidence along z."""
    pts = []
    for i in range(B):
        frac = 0.70 + 0.20 * (i // 2) / max(1, (B // 2) - 1)
        pol = (1.0, 0.0, 0.0) if i % 2 == 0 else (0.0, 1.0, 0.0)
        pts.append(point(frac * k0, (0.0, 0.0, 1.0), pol, k0))
    return pts
