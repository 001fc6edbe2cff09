"""The parameter studies of Figs. 4 and 5 through the CUDA path: symmetry of
the cubic point, parity with the oracle's retrieval, and the normal surface
against Fresnel's equation in the effective-medium limit."""
import math

import numpy as np
import pytest

from oracle import retrieval as ort
from paper_1501_01752_b300 import workloads as wl

from gpu_common import gsm

pytestmark = pytest.mark.gpu


def _st(periods, r):
    from paper_1501_01752_b300 import studies
    return studies.cavity_structure(periods, r)


def test_cubic_point_has_equal_principal_indices():
    # ratio 1: the cell is cubic, so the three principal sweeps are images of
    # each other under 90-degree rotations; finite period raises the index
    # above Maxwell-Garnett (Fig. 4a at ratio 1)
    g = gsm()
    from paper_1501_01752_b300 import studies
    r = 0.02
    P = studies.tetragonal_periods(1.0, r)
    n_mg = math.sqrt(studies.maxwell_garnett(1.0, 2.25, 4 * math.pi / 81))
    n = studies.principal_indices(_st(P, r), (7, 7, 7), n_mg, precision=g.FP64, tol=1e-12)
    assert np.max(n) - np.min(n) < 1e-7, n
    assert n_mg < n[0] < n_mg + 5e-3, (n, n_mg)


def test_tetragonal_indices_match_oracle():
    g = gsm()
    from paper_1501_01752_b300 import studies
    r = 0.03
    P = studies.tetragonal_periods(1.3, r)
    st = _st(P, r)
    n_mg = math.sqrt(studies.maxwell_garnett(1.0, 2.25, 4 * math.pi / 81))
    n = studies.principal_indices(st, (5, 5, 5), n_mg, precision=g.FP64, tol=1e-12)
    ost = ort.Structure(st["periods"], st["eps_host"], st["shapes"])
    kap = np.linspace(2 * math.pi * n_mg * 0.88, 2 * math.pi * n_mg * 1.12, 16)
    want = np.sqrt(ort.retrieve_tensor(ost, (5, 5, 5), 1.0, 2 * math.pi, [kap] * 3).real)
    assert np.max(np.abs(n - want)) < 1e-8, (n, want)


def test_normal_surface_matches_fresnel_in_effective_medium_limit():
    # small cavities (0.01 wavelengths): the off-axis mode indices lie on the
    # normal surface of the effective biaxial medium built from the three
    # principal indices; larger cavities depart from it (spatial dispersion)
    g = gsm()
    from paper_1501_01752_b300 import studies
    n_mg = math.sqrt(studies.maxwell_garnett(1.0, 2.25, 4 * math.pi / 81 / 1.1))
    thetas = (math.pi / 6, math.pi / 3)
    dev = {}
    for r in (0.01, 0.05):
        P = studies.orthorhombic_periods(1.3, r)
        st = _st(P, r)
        n = studies.principal_indices(st, (7, 7, 7), n_mg, precision=g.FP64, tol=1e-12)
        surf = studies.normal_surface_xz(st, (7, 7, 7), thetas, n_mg, precision=g.FP64, tol=1e-12)
        want = np.array([studies.fresnel_xz(n, t) for t in thetas])
        dev[r] = np.max(np.abs(surf - want))
    assert dev[0.01] < 2e-4, dev
    assert dev[0.01] < dev[0.05], dev


def test_figure_claims():
    # the section's statements, at 0.02-wavelength cavities and 9 harmonics:
    # ratio 1 lies above Maxwell-Garnett; the tetragonal lattice is uniaxial
    # (n_y = n_z) with one index below the MG line away from ratio 1; the
    # orthorhombic lattice has all three indices above MG at ratio 1 and two
    # below it at ratio 0.7
    g = gsm()
    from paper_1501_01752_b300 import studies
    kw = dict(precision=g.FP32_REFINE, tol=1e-10)
    fig4 = studies.figure("tetragonal", (9, 9, 9), ratios=(0.7, 1.0, 1.3), radii=(0.02,), **kw)
    n_mg = fig4["n_mg"]
    lo, mid, hi = (np.array(r["n"]) for r in fig4["rows"])
    assert np.all(mid > n_mg) and np.max(mid) - np.min(mid) < 1e-6
    for n in (lo, hi):
        assert abs(n[1] - n[2]) < 5e-5
    assert lo[1] < n_mg < lo[0] and hi[0] < n_mg < hi[1]
    fig5 = studies.figure("orthorhombic", (9, 9, 9), ratios=(0.7, 1.0), radii=(0.02,), **kw)
    n_mg5 = fig5["n_mg"]
    lo5, mid5 = (np.array(r["n"]) for r in fig5["rows"])
    assert np.all(mid5 > n_mg5)
    assert np.sum(lo5 < n_mg5) == 2
