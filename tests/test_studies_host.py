"""Host-side pieces of the parameter studies (no GPU): the fixed-fill
lattice geometry of the figures and Fresnel's equation."""
import math

import numpy as np

from paper_1501_01752_b300 import studies


def test_fixed_fill_geometry():
    for ratio in (0.7, 1.0, 1.3):
        for r in (0.01, 0.05):
            P = studies.tetragonal_periods(ratio, r)
            assert abs(P[1] - P[2]) < 1e-15 and abs(P[0] / P[2] - ratio) < 1e-12
            assert abs(4 * math.pi * r**3 / 3 / np.prod(P) - 0.155) < 1e-3
            Q = studies.orthorhombic_periods(ratio, r)
            assert abs(Q[1] / Q[2] - 1.1) < 1e-12 and abs(Q[0] / Q[2] - ratio) < 1e-12
            assert abs(4 * math.pi * r**3 / 3 / np.prod(Q) - 0.141) < 1e-3
    # the isotropic points: radius = Lambda / 3 (tetragonal), Lambda_x / 3 with Lambda_x = Lambda_z
    assert abs(studies.tetragonal_periods(1.0, 0.03)[0] - 0.09) < 1e-12
    assert abs(studies.orthorhombic_periods(1.0, 0.03)[0] - 0.09) < 1e-12


def test_maxwell_garnett_printed_values():
    # the figures' horizontal lines: 1.4213 (f = 0.155) and 1.4284 (f = 0.141)
    n4 = math.sqrt(studies.maxwell_garnett(1.0, 2.25, 4 * math.pi / 81))
    n5 = math.sqrt(studies.maxwell_garnett(1.0, 2.25, 4 * math.pi / 81 / 1.1))
    assert abs(n4 - 1.4213) < 1e-4 and abs(n5 - 1.4284) < 1e-4


def test_fresnel_xz_limits_and_ellipse():
    n = (1.40, 1.42, 1.45)
    o, e = studies.fresnel_xz(n, 0.0)
    assert o == 1.42 and abs(e - 1.40) < 1e-15
    o, e = studies.fresnel_xz(n, math.pi / 2)
    assert o == 1.42 and abs(e - 1.45) < 1e-15
    # the in-plane sheet is the ellipse x^2 / n_z^2 + z^2 / n_x^2 = 1 of (n sin t, n cos t)
    for t in np.linspace(0.1, 1.4, 5):
        _, e = studies.fresnel_xz(n, t)
        assert abs((e * math.sin(t))**2 / n[2]**2 + (e * math.cos(t))**2 / n[0]**2 - 1) < 1e-14
