"""Parity of the 128-point lane-team product (16-lane teams: N from 33 to 63
harmonics per axis on a cubic 128^3 grid) with the oracle's Eq. 4 and Eq. 5
operators, in FP64, complex64 and double-float, and a refined solve on that
grid checked by the oracle's residual."""
import numpy as np
import pytest

from oracle import operator as oop
from paper_1501_01752_b300 import workloads as wl

from gpu_common import K0, gsm, oracle_structure, rel

pytestmark = pytest.mark.gpu

CASES = [
    # (structure, n_harm, eps_b, points); every FFT size 128 unless noted
    ("woodpile_63", wl.woodpile(), (63, 63, 63), 1.0,
     [wl.point(0.8 * K0), wl.point(0.9 * K0, (0.6, 0, 0.8), (0, 1, 0))]),
    ("random_41", wl.random_shapes(6), (41, 41, 41), 1.3,
     [wl.point(0.71 * K0, (0.3, -0.2, 0.9), (0.2, 0.5, 0.1j))]),
    # unequal harmonic counts on the same grid: ragged rows in all passes
    ("random_33_47_63", wl.random_shapes(7, period=(0.3, 0.32, 0.34)), (33, 47, 63), 1.0,
     [wl.point(0.77 * K0, (0.2, 0.3, 0.9), (1, 0, 0.1))]),
    # 128 / 64 / 64: not a lane-team grid, the shared-memory path runs
    ("random_63_31_31", wl.random_shapes(8), (63, 31, 31), 1.0, [wl.point(0.8 * K0)]),
]
CUBIC = ("woodpile_63", "random_41", "random_33_47_63")


def _oracle_apply(st, n_harm, eps_b, pt, x, form):
    ost = oracle_structure(st)
    kinc = pt["kappa"] * np.asarray(pt["kdir"])
    kb2 = pt["k0"] ** 2 * eps_b
    if form == "H":
        return oop.OperatorH(ost.delta_h(n_harm, eps_b), n_harm, kinc, st["periods"], kb2)(x)
    return oop.Operator(ost.delta(n_harm, eps_b), n_harm, kinc, st["periods"], kb2)(x)


@pytest.mark.parametrize("form", ["E", "H"])
@pytest.mark.parametrize("name,st,n_harm,eps_b,points", CASES, ids=[c[0] for c in CASES])
def test_apply_128_matches_oracle(name, st, n_harm, eps_b, points, form):
    g = gsm()
    x = wl.random_field(n_harm, 700 + len(name), batch=len(points))
    plan = g.plan_for(st, n_harm, eps_b=eps_b, precision=g.FP32_REFINE,
                      form=g.FORM_H if form == "H" else g.FORM_E)
    y64 = plan.apply(points, x, precision=g.FP64)
    y32 = plan.apply(points, x, precision=g.FP32_REFINE)
    ydf = plan.apply(points, x, precision=g.DF64) if name in CUBIC else None
    for b, pt in enumerate(points):
        want = _oracle_apply(st, n_harm, eps_b, pt, x[b], form)
        assert rel(y64[b], want) < 1e-12, (name, form, b, rel(y64[b], want))
        assert rel(y32[b], want) < 1e-5, (name, form, b, rel(y32[b], want))
        if ydf is not None:
            assert rel(ydf[b], want) < 1e-12, (name, form, b, rel(ydf[b], want))
    plan.close()


def test_adjoint_128_matches_oracle():
    g = gsm()
    st = wl.random_shapes(6)
    n_harm = (41, 41, 41)
    pts = [wl.point(0.71 * K0, (0.3, -0.2, 0.9), (0.2, 0.5, 0.1j)), wl.point(1.1 * K0, (1, 0, 0), (0, 0, 1))]
    x = wl.random_field(n_harm, 77, batch=2)
    plan = g.plan_for(st, n_harm, eps_b=1.3, precision=g.FP32_REFINE)
    ost = oracle_structure(st)
    D = ost.delta(n_harm, 1.3)
    for prec, tol in ((g.FP64, 1e-12), (g.FP32_REFINE, 1e-5)):
        y = plan.apply(pts, x, precision=prec, adjoint=True)
        for b, pt in enumerate(pts):
            A = oop.Operator(D, n_harm, pt["kappa"] * np.asarray(pt["kdir"]), st["periods"], pt["k0"] ** 2 * 1.3)
            want = A.adjoint(x[b])
            assert rel(y[b], want) < tol, (prec, b, rel(y[b], want))
    plan.close()


@pytest.mark.parametrize("krylov", ["gmres", "bicgstab"])
def test_refined_solve_63_oracle_residual(krylov):
    g = gsm()
    st = wl.woodpile()
    n_harm = (63, 63, 63)
    pts = [wl.point(0.8 * K0), wl.point(0.75 * K0, (0, 0, 1), (0, 1, 0))]
    plan = g.plan_for(st, n_harm, precision=g.FP32_REFINE, tol=1e-8,
                      krylov=g.BICGSTAB if krylov == "bicgstab" else g.GMRES)
    E, infos, s = plan.solve(pts)
    assert s == 0
    D = oracle_structure(st).delta(n_harm, 1.0)
    U = 3 * 63 ** 3
    for b, p in enumerate(pts):
        A = oop.Operator(D, n_harm, p["kappa"] * np.asarray(p["kdir"]), st["periods"], p["k0"] ** 2)
        bvec = oop.incident(p["pol"], n_harm)
        res = np.linalg.norm(bvec - A(E[b * U:(b + 1) * U].reshape(bvec.shape))) / np.linalg.norm(bvec)
        assert res <= 1.5e-8, (b, res, infos[b])
    plan.close()
