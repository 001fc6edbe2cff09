"""Mixed-radix FFT sizes (L = 3 * 2^p: 24, 48, 96) in the product and the
solve, against the oracle: the cyclic convolution on any L >= 2N - 1 equals
the truncated Toeplitz product, so the answers must not depend on L."""
import numpy as np
import pytest

from oracle import operator as oop
from oracle import retrieval as ort
from paper_1501_01752_b300 import workloads as wl

from gpu_common import K0, gsm, oracle_structure, rel

pytestmark = pytest.mark.gpu

CASES = [
    ("ellipsoid_21_L48", wl.ellipsoid_lattice(), (21, 21, 21), (48, 48, 48)),
    ("random_11_L24", wl.random_shapes(2), (11, 11, 11), (24, 24, 24)),
    ("random_mixed_axes", wl.random_shapes(6, period=(0.3, 0.32, 0.34)), (41, 15, 21), (96, 32, 48)),
    ("woodpile_21_L48_64", wl.woodpile(), (21, 21, 21), (48, 64, 48)),
]


@pytest.mark.parametrize("name,st,n_harm,fft", CASES, ids=[c[0] for c in CASES])
def test_apply_on_mixed_grids_matches_oracle(name, st, n_harm, fft):
    g = gsm()
    pts = [wl.point(0.8 * K0), wl.point(0.73 * K0, (0.3, -0.2, 0.9), (0.2, 0.5, 0.1j))]
    x = wl.random_field(n_harm, 700 + len(name), batch=len(pts))
    ost = oracle_structure(st)
    Delta = ost.delta(n_harm, 1.0)
    plan = g.plan_for(st, n_harm, precision=g.FP64, fft=fft)
    assert g.plan_query(st["periods"], n_harm, fft=fft)[0] == tuple(fft)
    for adjoint in (False, True):
        y64 = plan.apply(pts, x, precision=g.FP64, adjoint=adjoint)
        y32 = plan.apply(pts, x, precision=g.FP32_REFINE, adjoint=adjoint)
        for b, p in enumerate(pts):
            A = oop.Operator(Delta, n_harm, p["kappa"] * np.asarray(p["kdir"]), st["periods"], p["k0"] ** 2)
            want = A.adjoint(x[b]) if adjoint else A(x[b])
            assert rel(y64[b], want) < 1e-12, (name, adjoint, b, rel(y64[b], want))
            assert rel(y32[b], want) < 1e-5, (name, adjoint, b, rel(y32[b], want))
    plan.close()
    # the H-field form on the same grids
    plan = g.plan_for(st, n_harm, precision=g.FP64, fft=fft, form=g.FORM_H)
    y = plan.apply(pts, x, precision=g.FP64)
    Dh = ost.delta_h(n_harm, 1.0)
    for b, p in enumerate(pts):
        A = oop.OperatorH(Dh, n_harm, p["kappa"] * np.asarray(p["kdir"]), st["periods"], p["k0"] ** 2)
        assert rel(y[b], A(x[b])) < 1e-12
    plan.close()


@pytest.mark.parametrize("krylov", ["gmres", "bicgstab"])
def test_refined_solve_on_L48_matches_power_of_two_grid(krylov):
    g = gsm()
    st = wl.ellipsoid_lattice()
    n_harm = (21, 21, 21)
    pts = [wl.point((0.7 + 0.05 * i) * K0, (0, 0, 1), (1, 0, 0) if i % 2 == 0 else (0, 1, 0)) for i in range(4)]
    kr = g.BICGSTAB if krylov == "bicgstab" else g.GMRES
    p48 = g.plan_for(st, n_harm, precision=g.FP32_REFINE, tol=1e-10, fft=(48, 48, 48), krylov=kr)
    E48, i48, s48 = p48.solve(pts)
    p48.close()
    p64 = g.plan_for(st, n_harm, precision=g.FP32_REFINE, tol=1e-10, krylov=kr)
    E64, _, s64 = p64.solve(pts)
    p64.close()
    assert s48 == 0 and s64 == 0
    assert rel(E48, E64) < 1e-8
    U = 3 * 21 ** 3
    ost = oracle_structure(st)
    E, _ = ort.solve_point(ost, n_harm, 1.0, pts[0]["k0"], pts[0]["kdir"], pts[0]["kappa"], pts[0]["pol"], tol=1e-12)
    assert rel(E48[:U], E.ravel()) < 1e-8


def test_tuned_grid_choice_and_solution():
    # fft = -1: each level times one product on the power-of-two grid and on
    # the smaller mixed-radix one and keeps the faster; the fields do not
    # depend on the choice, and the choice survives a new permittivity
    g = gsm()
    st = wl.ellipsoid_lattice()
    pts = [wl.point((0.7 + 0.05 * i) * K0, (0, 0, 1), (1, 0, 0)) for i in range(4)]
    ost = oracle_structure(st)
    for N, cands in ((21, ((48,) * 3, (64,) * 3)), (41, ((96,) * 3, (128,) * 3))):
        n_harm = (N, N, N)
        plan = g.plan_for(st, n_harm, precision=g.FP32_REFINE, tol=1e-8, fft=(-1, -1, -1), max_batch=4)
        with pytest.raises(g.GsmError):
            plan.level_fft((9, 9, 9))              # a truncation no call has used yet
        E, infos, s = plan.solve(pts)
        L = plan.level_fft(n_harm)
        assert s == 0 and L in cands, L
        Delta = ost.delta(n_harm, 1.0)
        U = 3 * N ** 3
        for b, p in enumerate(pts[:2]):
            A = oop.Operator(Delta, n_harm, p["kappa"] * np.asarray(p["kdir"]), st["periods"], p["k0"] ** 2)
            bv = oop.incident(p["pol"], n_harm)
            res = np.linalg.norm(bv - A(E[b * U:(b + 1) * U].reshape(bv.shape))) / np.linalg.norm(bv)
            assert res <= 1.5e-8, (N, b, res)
        plan.set_structure(wl.ellipsoid_lattice(eps=5.0))
        plan.solve(pts[:1])
        assert plan.level_fft(n_harm) == L
        plan.close()
