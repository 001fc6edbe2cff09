"""Pins for oracle.coefficients: Fourier images of the permittivity
("Calculation details": analytic images of simple shapes, combined)."""
import numpy as np
import pytest
from scipy import integrate

from oracle import coefficients as co

V = 0.3 * 0.33 * 0.36


def test_sphere_image_equals_radial_quadrature():
    # chi(G) = V^-1 4 pi \int_0^R r^2 sin(G r)/(G r) dr: the angular integral
    # of exp(-i G.r) over a sphere done analytically, the radial one numerically.
    R = 0.11
    for G in [0.0, 3.0, 21.0, 57.5, 140.0]:
        if G == 0.0:
            ref = 4 * np.pi * R**3 / 3 / V
        else:
            ref = 4 * np.pi * integrate.quad(lambda r: r * np.sin(G * r) / G, 0, R,
                                             epsabs=1e-15, epsrel=1e-13, limit=200)[0] / V
        got = co.shape_image(co.SPHERE, (R, 0, 0), G, 0.0, 0.0, V)
        assert abs(got - ref) < 1e-12, (G, got, ref)
        # isotropy: the same |G| along another direction
        got2 = co.shape_image(co.SPHERE, (R, 0, 0), G / np.sqrt(3), G / np.sqrt(3), G / np.sqrt(3), V)
        assert abs(got2 - ref) < 1e-12


def test_box_equals_exactly_voxelised_box():
    # A box whose faces lie on voxel boundaries: the analytic sinc-product image
    # (with the exp(-i G.c) centre phase) must equal the exact voxel integral.
    periods = (0.3, 0.33, 0.36)
    M = (8, 10, 12)  # (Mx, My, Mz)
    lo, hi = (2, 3, 1), (5, 9, 12)
    eps_h, eps_s = 1.7, 6.5
    vox = np.full((M[2], M[1], M[0]), eps_h)
    vox[lo[2]:hi[2], lo[1]:hi[1], lo[0]:hi[0]] = eps_s
    h = [periods[a] / M[a] for a in range(3)]
    center = tuple((lo[a] + hi[a]) / 2 * h[a] for a in range(3))
    size = tuple((hi[a] - lo[a]) * h[a] for a in range(3))
    dmax = (9, 7, 13)
    ref = co.voxel_coefficients(vox, dmax)
    got = co.shapes_coefficients(eps_h, [(co.BOX, center, size, eps_s)], periods, dmax)
    assert np.max(np.abs(got - ref)) < 1e-13


def test_single_voxel_equals_quadrature():
    # one voxel of value 1 at v = (3, 1, 4) in a (5, 6, 7) grid: each 1D factor
    # V_a^-1 \int exp(-i d K x) dx over the voxel, integrated numerically.
    periods = (1.0, 1.0, 1.0)
    M = (5, 6, 7)
    v = (3, 1, 4)
    vox = np.zeros((M[2], M[1], M[0]))
    vox[v[2], v[1], v[0]] = 1.0
    dmax = (4, 3, 5)
    got = co.voxel_coefficients(vox, dmax)

    def factor(d, a):
        x0, x1 = v[a] / M[a], (v[a] + 1) / M[a]
        K = 2 * np.pi * d
        re = integrate.quad(lambda x: np.cos(K * x), x0, x1, epsabs=1e-15)[0]
        im = integrate.quad(lambda x: -np.sin(K * x), x0, x1, epsabs=1e-15)[0]
        return re + 1j * im

    for dz in (-5, 0, 2, 5):
        for dy in (-3, 1):
            for dx in (-4, 0, 3):
                ref = factor(dx, 0) * factor(dy, 1) * factor(dz, 2)
                assert abs(got[dz + 5, dy + 3, dx + 4] - ref) < 1e-14


def test_ellipsoid_brute_force_and_sphere_limit():
    semi = (0.12, 0.09, 0.06)
    periods = (0.3, 0.33, 0.36)
    G = (2 * np.pi / periods[0] * 1, 2 * np.pi / periods[1] * -2, 2 * np.pi / periods[2] * 1)
    got = co.shape_image(co.ELLIPSOID, semi, *G, V)
    # midpoint-rule quadrature of the indicator on a fine grid (O(h) accurate)
    n = 160
    xs = [(np.arange(n) + 0.5) / n * 2 * s - s for s in semi]
    Z, Y, X = np.meshgrid(xs[2], xs[1], xs[0], indexing="ij")
    inside = (X / semi[0])**2 + (Y / semi[1])**2 + (Z / semi[2])**2 <= 1.0
    dv = np.prod([2 * s / n for s in semi])
    ref = np.sum(np.exp(-1j * (G[0] * X + G[1] * Y + G[2] * Z))[inside]) * dv / V
    f = 4 * np.pi * np.prod(semi) / 3 / V
    assert abs(got - ref) < 5e-3 * f
    # semi-axes all equal: the sphere image
    s = co.shape_image(co.ELLIPSOID, (0.1, 0.1, 0.1), *G, V)
    r = co.shape_image(co.SPHERE, (0.1, 0, 0), *G, V)
    assert abs(s - r) < 1e-15


def test_mean_is_volume_average_and_real_eps_is_hermitian():
    from paper_1501_01752_b300 import workloads as wl
    w = wl.woodpile()
    dmax = (6, 6, 6)
    eps = co.shapes_coefficients(w["eps_host"], w["shapes"], w["periods"], dmax)
    assert abs(eps[6, 6, 6] - (1.0 + 0.25 * (11.9 - 1.0))) < 1e-13   # fill 0.25
    # real eps(r) => eps_{-d} = conj(eps_d)
    assert np.max(np.abs(eps[::-1, ::-1, ::-1] - np.conj(eps))) < 1e-14
    # rods spanning the period along x (resp. y) have no x (resp. y) harmonics
    # except where the other rod contributes: the x-rod alone
    x_rod = [w["shapes"][0]]
    e1 = co.shapes_coefficients(1.0, x_rod, w["periods"], dmax)
    assert np.max(np.abs(e1[:, :, np.arange(13) != 6])) < 1e-15


def test_delta_coefficients():
    eps = np.zeros((3, 3, 3), complex)
    eps[1, 1, 1] = 4.0
    eps[0, 1, 2] = 0.5 - 0.25j
    d = co.delta_coefficients(eps, 2.0)
    assert d[1, 1, 1] == 1.0 and d[0, 1, 2] == 0.25 - 0.125j
