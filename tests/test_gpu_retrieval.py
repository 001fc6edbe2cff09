"""Effective-tensor retrieval through the CUDA sweep + host pole fit, against
the closed form (homogeneous medium) and the oracle's retrieval."""
import numpy as np
import pytest

from oracle import retrieval as ort
from paper_1501_01752_b300 import workloads as wl

from gpu_common import K0, gsm, oracle_structure

pytestmark = pytest.mark.gpu


def _windows(n_centre, rel=0.15):
    """kappa intervals around k0 n_centre that keep clear of the basis light
    cone kappa = k0 (eps_b = 1), where Eq. 4 is singular at m = 0."""
    w = []
    for n in np.broadcast_to(n_centre, 3):
        lo = max(K0 * n * (1 - rel), 1.03 * K0) if n > 1 else K0 * n * (1 - rel)
        w.append((lo, K0 * n * (1 + rel)))
    return np.array(w)


def test_homogeneous_medium_exact_index():
    g = gsm()
    st = dict(periods=(0.3, 0.31, 0.32), eps_host=2.25, shapes=[])
    plan = g.plan_for(st, (3, 3, 3), precision=g.FP64, tol=1e-12)
    eps, diag = plan.retrieve_tensor(K0, _windows(1.5), n_kappa=16)
    assert np.max(np.abs(eps - 2.25)) < 1e-9, eps
    eta = diag["eta"][0]
    assert abs(diag["zeta"][0] - (eta**2 - K0**2) / (2 * eta)) < 1e-6
    plan.close()


@pytest.mark.parametrize("name,st,prec", [
    ("spheres_fp64", wl.sphere_lattice(), "fp64"),
    ("spheres_fp32", wl.sphere_lattice(), "fp32"),
    ("ellipsoids_fp64", wl.ellipsoid_lattice(), "fp64"),
])
def test_retrieval_matches_oracle(name, st, prec):
    g = gsm()
    n_harm = (7, 7, 7)
    f = sum(4 / 3 * np.pi * np.prod(s[2] if s[0] == wl.ELLIPSOID else (s[2][0],) * 3) for s in st["shapes"]) / np.prod(st["periods"])
    n_mg = np.sqrt(ort.maxwell_garnett(st["shapes"][0][3], 1.0, f))
    win = _windows(n_mg, 0.2)
    fp64 = prec == "fp64"
    plan = g.plan_for(st, n_harm, precision=g.FP64 if fp64 else g.FP32_REFINE, tol=1e-12 if fp64 else 1e-10)
    eps, diag = plan.retrieve_tensor(K0, win, n_kappa=16)
    plan.close()
    ost = oracle_structure(st)
    ref = ort.retrieve_tensor(ost, n_harm, 1.0, K0, [np.linspace(lo, hi, 16) for lo, hi in win], method="lu")
    assert np.max(np.abs(eps - ref.real) / ref.real) < 1e-6, (eps, ref)
    if name.startswith("ellipsoids"):
        assert eps[0] > eps[1] > eps[2] > 1.0     # semi-axes 0.4 > 0.3 > 0.2: biaxial ordering
