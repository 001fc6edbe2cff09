"""CUDA adjoint gradients with respect to voxel permittivity against the
oracle's explicit adjoint and against central finite differences."""
import numpy as np
import pytest

from oracle import adjoint as oadj
from oracle import retrieval as ort
from paper_1501_01752_b300 import workloads as wl

from gpu_common import K0, gsm, rel

pytestmark = pytest.mark.gpu


def _vox(seed, M=8, fill=0.3):
    rng = np.random.default_rng(seed)
    return np.where(rng.random((M, M, M)) < fill, 6.0, 1.0)


@pytest.mark.parametrize("prec", ["fp64", "c64_refine"])
def test_xi_gradient_matches_oracle(prec):
    g = gsm()
    vox = _vox(1)
    periods = (0.3, 0.3, 0.3)
    n_harm = (5, 5, 5)
    st = dict(periods=periods, voxels=vox)
    pts = [wl.point(0.9 * K0), wl.point(0.95 * K0, (0, 0, 1), (0, 1, 0)), wl.point(0.85 * K0, (1, 0, 0), (0, 0, 1))]
    fp64 = prec == "fp64"
    plan = g.plan_for(st, n_harm, precision=g.FP64 if fp64 else g.FP32_REFINE, tol=1e-13 if fp64 else 1e-11)
    ost = ort.Structure(periods, voxels=vox)
    # objective L = sum_i Re(conj(c_i) xi_i), xi_i = a_i^H E_0: gradient wrt E_0 is c_i a_i
    cs = [1.0, 0.5 - 0.25j, -0.7j]
    gE0 = np.array([c * np.asarray(p["pol"]) for c, p in zip(cs, pts)])
    got = plan.adjoint(pts, gE0)
    want = np.zeros_like(vox)
    for c, p in zip(cs, pts):
        _, dxi = oadj.xi_voxel_gradient(ost, n_harm, 1.0, p["k0"], p["kdir"], p["kappa"], p["pol"], tol=1e-13)
        want += (np.conj(c) * dxi).real
    assert rel(got, want) < (1e-8 if fp64 else 1e-6), rel(got, want)
    plan.close()


def test_tensor_gradient_matches_oracle_and_finite_differences():
    # mirror-symmetric cell: principal axes along x, y, z as the retrieval assumes
    g = gsm()
    vox = wl.random_binary_voxels(M=8, seed=2, sigma=1.0, fill=0.25, mirror=True)
    periods = (0.25, 0.25, 0.25)
    n_harm = (5, 5, 5)
    st = dict(periods=periods, voxels=vox)
    f = float(np.mean(vox > 2))
    n0 = np.sqrt(ort.maxwell_garnett(6.0, 1.0, f))
    win = np.array([(K0 * n0 * 0.85, K0 * n0 * 1.15)] * 3)
    plan = g.plan_for(st, n_harm, precision=g.FP64, tol=1e-13)
    weights = (1.0, -1.0, 0.0)
    eps, grad = plan.retrieve_tensor_grad(K0, win, weights, n_kappa=16)
    ost = ort.Structure(periods, voxels=vox)
    kap = np.linspace(win[0][0], win[0][1], 16)
    exx, gxx = oadj.component_gradient(ost, n_harm, 1.0, K0, (0, 0, 1), (1, 0, 0), kap)
    eyy, gyy = oadj.component_gradient(ost, n_harm, 1.0, K0, (0, 0, 1), (0, 1, 0), kap)
    assert abs(eps[0] - exx.real) < 1e-8 and abs(eps[1] - eyy.real) < 1e-8
    assert rel(grad, gxx - gyy) < 1e-5, rel(grad, gxx - gyy)
    # central differences of the CUDA retrieval itself
    h = 1e-3
    for v in [(0, 0, 0), (3, 5, 1), (7, 2, 6)]:
        vals = []
        for sgn in (1, -1):
            vv = vox.copy()
            vv[v] += sgn * h
            plan.set_permittivity(voxels=vv)
            e, _ = plan.retrieve_tensor(K0, win, n_kappa=16)
            vals.append(e[0] - e[1])
        fd = (vals[0] - vals[1]) / (2 * h)
        assert abs(fd - grad[v]) < 1e-5 * max(1e-3, np.max(np.abs(grad))), (v, fd, grad[v])
    plan.close()
