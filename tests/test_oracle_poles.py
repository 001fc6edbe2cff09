"""Pins for oracle.poles (Eqs. 6-10) and the Maxwell-Garnett helper."""
import json
import os

import numpy as np

from oracle import poles
from oracle import retrieval as rt

K0 = 2 * np.pi
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")


def test_divided_difference_of_polynomials():
    # textbook: the order-n divided difference of a degree-n polynomial is its
    # leading coefficient, and of any lower degree polynomial it is zero.
    t = np.linspace(-1, 1, 11) + 0.01 * np.sin(np.arange(11))
    c = poles.dd_weights(t)
    assert abs(np.sum(c * (3.0 * t**10 - 2 * t**3 + 1)) - 3.0) < 1e-9
    for deg in range(10):
        assert abs(np.sum(c * t**deg)) < 1e-9


def test_fit_recovers_synthetic_meromorphic_function():
    # xi = sum_j zeta_j/(kappa-eta_j) + gamma_0 + gamma_1 kappa (Eq. 6 truncated):
    # P xi is a polynomial of degree <= Np + 1 < Nd, so Eq. 8 holds exactly.
    kap = np.linspace(9.0, 11.0, 16)
    eta = np.array([10.13 + 0.0j, 12.9 - 0.4j])
    zeta = np.array([0.7 + 0.0j, -1.3 + 0.2j])
    xi = sum(z / (kap - e) for z, e in zip(zeta, eta)) + 0.3 - 0.05 * kap
    e, z = poles.fit_poles(kap, xi, Np=5, Nd=10)
    for ej, zj in zip(eta, zeta):
        k = np.argmin(np.abs(e - ej))
        assert abs(e[k] - ej) < 1e-9 and abs(z[k] - zj) < 1e-8
    # the three spurious roots carry no residue
    keep = [np.argmin(np.abs(e - ej)) for ej in eta]
    spurious = np.delete(z, keep)
    assert np.max(np.abs(spurious)) < 1e-8
    j = poles.select_pole(e, z, kap.min(), kap.max())
    assert abs(e[j] - eta[0]) < 1e-9


def test_fit_exact_with_np_poles():
    kap = np.linspace(-1.0, 1.0, 15)
    eta = np.array([0.1, -0.45 + 0.3j, 0.8 - 0.2j, 1.7, -2.2j])
    zeta = np.array([1.0, 0.2j, -0.5, 3.0, 0.1 + 0.1j])
    xi = sum(z / (kap - e) for z, e in zip(zeta, eta))
    e, z = poles.fit_poles(kap, xi, Np=5, Nd=10)
    order = [int(np.argmin(np.abs(e - ej))) for ej in eta]
    # poles near the nodes are fixed to roundoff; the ones far outside
    # [-1, 1] (1.7, -2.2i) are conditioned ~|eta|^Nd worse
    near = np.abs(eta) < 1.0
    assert np.max(np.abs(e[order] - eta)[near]) < 1e-12
    assert np.max(np.abs(z[order] - zeta)[near]) < 1e-11
    assert np.max(np.abs(e[order] - eta)) < 1e-6
    assert np.max(np.abs(z[order] - zeta)) < 1e-5


def test_pole_gradient_matches_finite_differences():
    # one pole in the window plus a regular part that is not a low-degree
    # polynomial (more far poles than Np); perturbations the model represents:
    # moving the pole, changing its residue, changing the regular part.
    kap = np.linspace(9.0, 11.0, 16)

    def make(eta0=10.13, z0=0.7, g0=0.3):
        xi = z0 / (kap - eta0) + g0 - 0.05 * kap
        for e_far, z_far in ((13.0, 0.4), (6.5, -0.3), (15.0, 1.1), (4.0, 0.8), (17.0, -2.0)):
            xi = xi + z_far / (kap - e_far)
        return xi + 0j

    xi = make()
    e, z = poles.fit_poles(kap, xi, 5, 10)
    j = poles.select_pole(e, z, 9, 11)
    d_re, d_im = poles.pole_gradient(kap, xi, 5, 10, j)
    h = 1e-5
    for kw in (dict(eta0=10.13), dict(z0=0.7), dict(g0=0.3)):
        (name, v0), = kw.items()
        xp, xm = make(**{name: v0 + h}), make(**{name: v0 - h})
        ep, _ = poles.fit_poles(kap, xp, 5, 10)
        em, _ = poles.fit_poles(kap, xm, 5, 10)
        fd = (ep[np.argmin(abs(ep - e[j]))] - em[np.argmin(abs(em - e[j]))]) / (2 * h)
        dxi = (xp - xm) / (2 * h)
        lin = np.sum(d_re * dxi.real + d_im * dxi.imag)
        assert abs(fd - lin) < 1e-7, (name, fd, lin)
    assert abs(np.sum(d_re * ((make(10.13 + h) - make(10.13 - h)) / (2 * h)).real) - 1.0) < 1e-7


def test_maxwell_garnett_printed_values():
    # the paper prints n_MG = 1.4213 (f = 0.155) and 1.4284 (f = 0.141) for air
    # spheres of radius Lambda_x/3 in n = 1.5; f follows from the geometry.
    gold = json.load(open(GOLDEN))["maxwell_garnett"]
    for g in gold:
        f = 4 * np.pi / 3 * g["radius_over_period"]**3 / g["period_ratio_y"]
        assert abs(f - g["fill_printed"]) < 5e-4
        n = np.sqrt(rt.maxwell_garnett(g["eps_incl"], g["n_host"]**2, f))
        assert abs(n - g["n_MG_printed"]) < 0.5 * 10**-g["digits"], (n, g)
    # dilute limit: eps_MG = eps_h + 3 f eps_h beta + O(f^2)
    b = (6.0 - 1.0) / (6.0 + 2.0)
    assert abs(rt.maxwell_garnett(6.0, 1.0, 1e-6) - (1 + 3e-6 * b)) < 1e-11
