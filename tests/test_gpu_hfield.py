"""The H-field formulation (Eq. 5) in the CUDA path against the oracle's
Eq. 5 operator, its dense-LU solutions, its residual of the returned fields
and its H-form retrieval."""
import numpy as np
import pytest

from oracle import operator as oop
from oracle import retrieval as ort
from paper_1501_01752_b300 import workloads as wl

from gpu_common import K0, gsm, oracle_structure, rel

pytestmark = pytest.mark.gpu

CASES = [
    ("sphere_7", wl.sphere_lattice(), (7, 7, 7), 1.0, [wl.point(0.8 * K0, (0, 0, 1), (0, 1, 0))]),
    ("random_aniso", wl.random_shapes(1), (5, 9, 3), 1.3,
     [wl.point(0.71 * K0, (0.3, -0.2, 0.9), (0.2, 0.5, 0.1j)), wl.point(1.3 * K0, (1, 0, 0), (0, 1, 0))]),
    ("woodpile_15", wl.woodpile(), (15, 15, 15), 1.0,
     [wl.point(0.8 * K0, (0, 0, 1), (0, 1, 0)), wl.point(0.9 * K0, (0.6, 0, 0.8), (0, 1, 0))]),
    ("random_15_21_31", wl.random_shapes(4, period=(0.3, 0.32, 0.34)), (15, 21, 31), 1.0,
     [wl.point(0.77 * K0, (0.2, 0.3, 0.9), (1, 0, 0.1))]),
    ("woodpile_31", wl.woodpile(), (31, 31, 31), 1.0, [wl.point(0.8 * K0, (0, 0, 1), (0, 1, 0))]),
]


def _oracle_apply_h(st, n_harm, eps_b, pt, x):
    Dh = oracle_structure(st).delta_h(n_harm, eps_b)
    kinc = pt["kappa"] * np.asarray(pt["kdir"])
    return oop.OperatorH(Dh, n_harm, kinc, st["periods"], pt["k0"] ** 2 * eps_b)(x)


def _reg(n_harm):
    return all((2 ** int(np.ceil(np.log2(2 * N - 1)))) in (32, 64) for N in n_harm)


@pytest.mark.parametrize("path", ["auto", "team"])
@pytest.mark.parametrize("name,st,n_harm,eps_b,points", CASES, ids=[c[0] for c in CASES])
def test_apply_h_matches_oracle(name, st, n_harm, eps_b, points, path, monkeypatch):
    if path == "team":
        monkeypatch.setenv("GSM_FFT_PATH", "team")
    g = gsm()
    x = wl.random_field(n_harm, 500 + len(name), batch=len(points))
    plan = g.plan_for(st, n_harm, eps_b=eps_b, precision=g.FP64, form=g.FORM_H)
    y64 = plan.apply(points, x, precision=g.FP64)
    y32 = plan.apply(points, x, precision=g.FP32_REFINE)
    ydf = plan.apply(points, x, precision=g.DF64) if (path == "auto" and _reg(n_harm)) else None
    for b, pt in enumerate(points):
        want = _oracle_apply_h(st, n_harm, eps_b, pt, x[b])
        assert rel(y64[b], want) < 1e-12, (name, b, rel(y64[b], want))
        assert rel(y32[b], want) < 1e-5, (name, b, rel(y32[b], want))
        if ydf is not None:
            assert rel(ydf[b], want) < 1e-12, (name, b, rel(ydf[b], want))
    plan.close()


@pytest.mark.parametrize("prec,krylov", [("fp64", "gmres"), ("fp32", "gmres"), ("fp32", "bicgstab")])
def test_solve_h_matches_dense_lu(prec, krylov):
    g = gsm()
    st = wl.sphere_lattice()
    n_harm = (7, 7, 7)
    pts = [wl.point(0.8 * K0, (0, 0, 1), (0, 1, 0)), wl.point(0.7 * K0, (1, 1, 0), (0, 0, 1)),
           wl.point(1.05 * K0, (0, 0, 1), (1, 0, 0))]
    fp64 = prec == "fp64"
    plan = g.plan_for(st, n_harm, precision=g.FP64 if fp64 else g.FP32_REFINE, tol=1e-12 if fp64 else 1e-8,
                      form=g.FORM_H, krylov=g.BICGSTAB if krylov == "bicgstab" else g.GMRES)
    E, infos, s = plan.solve(pts)
    assert s == 0
    ost = oracle_structure(st)
    off = 0
    for b, p in enumerate(pts):
        U = plan.field_size(p)
        H, _ = ort.solve_point(ost, n_harm, 1.0, p["k0"], p["kdir"], p["kappa"], p["pol"], method="lu", form="H")
        assert rel(E[off:off + U], H.ravel()) < (1e-10 if fp64 else 1e-6), (b, rel(E[off:off + U], H.ravel()))
        off += U
    plan.close()


def test_solve_h_woodpile_31_refined_oracle_residual():
    g = gsm()
    st = wl.woodpile()
    n_harm = (31, 31, 31)
    pts = [wl.point(0.8 * K0, (0, 0, 1), (0, 1, 0)), wl.point(0.75 * K0, (0, 0, 1), (1, 0, 0))]
    plan = g.plan_for(st, n_harm, precision=g.FP32_REFINE, tol=1e-8, form=g.FORM_H)
    E, infos, s = plan.solve(pts)
    assert s == 0
    Dh = oracle_structure(st).delta_h(n_harm, 1.0)
    U = 3 * 31 ** 3
    for b, p in enumerate(pts):
        A = oop.OperatorH(Dh, n_harm, p["kappa"] * np.asarray(p["kdir"]), st["periods"], p["k0"] ** 2)
        bvec = oop.incident(p["pol"], n_harm)
        res = np.linalg.norm(bvec - A(E[b * U:(b + 1) * U].reshape(bvec.shape))) / np.linalg.norm(bvec)
        assert res <= 1.5e-8, (b, res, infos[b])
    plan.close()


def test_retrieve_tensor_h_matches_oracle():
    # the principal sweeps by their H polarisation; the pole of the same mode
    g = gsm()
    st = wl.ellipsoid_lattice(period=0.3)
    n_harm = (5, 5, 5)
    f = 4 * np.pi * 0.4 * 0.3 * 0.2 / 3
    n0 = np.sqrt(ort.maxwell_garnett(6.0, 1.0, f))
    win = np.array([(K0 * n0 * 0.85, K0 * n0 * 1.15)] * 3)
    plan = g.plan_for(st, n_harm, precision=g.FP64, tol=1e-12, form=g.FORM_H)
    eps, _ = plan.retrieve_tensor(K0, win, n_kappa=16)
    plan.close()
    ost = oracle_structure(st)
    want = ort.retrieve_tensor(ost, n_harm, 1.0, K0, [np.linspace(w[0], w[1], 16) for w in win], form="H")
    assert np.max(np.abs(eps - want.real)) < 1e-8, (eps, want)


def test_adjoint_is_refused_for_h():
    g = gsm()
    rng = np.random.default_rng(5)
    vox = np.where(rng.random((8, 8, 8)) < 0.3, 6.0, 1.0)
    st = dict(periods=(0.3, 0.3, 0.3), voxels=vox)
    plan = g.plan_for(st, (5, 5, 5), precision=g.FP64, form=g.FORM_H)
    with pytest.raises(g.GsmError) as ei:
        plan.adjoint([wl.point(0.9 * K0)], np.array([[1.0, 0, 0]]))
    assert ei.value.status == g.GSM_ERR_ARG
    x = wl.random_field((5, 5, 5), 1)
    with pytest.raises(g.GsmError) as ei:
        plan.apply([wl.point(0.9 * K0)], x[None], adjoint=True)
    assert ei.value.status == g.GSM_ERR_ARG
    plan.close()
