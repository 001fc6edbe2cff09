"""Parity of the CUDA Eq. 4 operator (three fused FFT passes + Green tensor)
with the oracle's operator, element by element on seeded inputs."""
import numpy as np
import pytest

from oracle import operator as oop
from paper_1501_01752_b300 import workloads as wl

from gpu_common import K0, gsm, oracle_structure, rel

pytestmark = pytest.mark.gpu

CASES = [
    # (structure, n_harm, eps_b, points)
    ("sphere_c1", wl.sphere_lattice(), (7, 7, 7), 1.0,
     [wl.point(0.8 * K0)]),
    ("random_aniso", wl.random_shapes(1), (5, 9, 3), 1.3,
     [wl.point(0.71 * K0, (0.3, -0.2, 0.9), (0.2, 0.5, 0.1j)), wl.point(1.3 * K0, (1, 0, 0), (0, 1, 0))]),
    ("layered_1d", wl.layered_stack(0.15, 0.5, 1.0, 4.0), (1, 1, 9), 1.0,
     [wl.point(1.2 * K0), wl.point(1.1 * K0, (1, 0, 0), (0, 0, 1))]),
    ("woodpile_15", wl.woodpile(), (15, 15, 15), 1.0,
     [wl.point(0.8 * K0), wl.point(0.75 * K0, (0, 0, 1), (0, 1, 0)), wl.point(0.9 * K0, (0.6, 0, 0.8), (0, 1, 0))]),
    ("ellipsoid_21", wl.ellipsoid_lattice(), (21, 21, 21), 1.0, [wl.point(0.83 * K0)]),
    ("woodpile_31", wl.woodpile(), (31, 31, 31), 1.0, [wl.point(0.8 * K0), wl.point(0.7 * K0, (0, 0, 1), (0, 1, 0))]),
    # mixed FFT sizes 32/64 per axis (register-FFT path with unequal axes)
    ("random_15_21_31", wl.random_shapes(4, period=(0.3, 0.32, 0.34)), (15, 21, 31), 1.0,
     [wl.point(0.77 * K0, (0.2, 0.3, 0.9), (1, 0, 0.1))]),
    ("random_21_15_15", wl.random_shapes(5), (21, 15, 15), 1.0, [wl.point(0.8 * K0)]),
]


def _oracle_apply(st, n_harm, eps_b, pt, x, adjoint):
    ost = oracle_structure(st)
    Delta = ost.delta(n_harm, eps_b)
    kinc = pt["kappa"] * np.asarray(pt["kdir"])
    A = oop.Operator(Delta, n_harm, kinc, st["periods"], pt["k0"] ** 2 * eps_b)
    return A.adjoint(x) if adjoint else A(x)


@pytest.mark.parametrize("path", ["auto", "team"])
@pytest.mark.parametrize("name,st,n_harm,eps_b,points", CASES, ids=[c[0] for c in CASES])
def test_apply_matches_oracle(name, st, n_harm, eps_b, points, path, monkeypatch):
    # "auto" takes the register-FFT kernels for complex64 when every FFT size is
    # 32 or 64; "team" forces the shared-memory FFT kernels everywhere
    if path == "team":
        monkeypatch.setenv("GSM_FFT_PATH", "team")
    g = gsm()
    x = wl.random_field(n_harm, 100 + len(name), batch=len(points))
    plan = g.plan_for(st, n_harm, eps_b=eps_b, precision=g.FP64)
    for adjoint in (False, True):
        y64 = plan.apply(points, x, precision=g.FP64, adjoint=adjoint)
        y32 = plan.apply(points, x, precision=g.FP32_REFINE, adjoint=adjoint)
        for b, pt in enumerate(points):
            want = _oracle_apply(st, n_harm, eps_b, pt, x[b], adjoint)
            assert rel(y64[b], want) < 1e-12, (name, adjoint, b, rel(y64[b], want))
            assert rel(y32[b], want) < 1e-5, (name, adjoint, b, rel(y32[b], want))
    plan.close()


def test_apply_on_device_tensors_and_linearity():
    import torch
    g = gsm()
    st = wl.woodpile()
    n_harm = (9, 11, 13)
    pts = [wl.point(0.8 * K0), wl.point(0.77 * K0, (0, 0, 1), (0, 1, 0))]
    plan = g.plan_for(st, n_harm, precision=g.FP64)
    x1 = wl.random_field(n_harm, 1, batch=2)
    x2 = wl.random_field(n_harm, 2, batch=2)
    y1 = plan.apply(pts, x1)
    yd = plan.apply(pts, torch.from_numpy(2 * x1 - 3j * x2).cuda()).cpu().numpy()
    y2 = plan.apply(pts, x2)
    assert rel(yd, 2 * y1 - 3j * y2) < 1e-13
    # the adjoint is the adjoint: <A x, y> = <x, A^H y>
    ax = plan.apply(pts, x1)
    ahy = plan.apply(pts, x2, adjoint=True)
    for b in range(2):
        lhs, rhs = np.vdot(x2[b], ax[b]), np.vdot(ahy[b], x1[b])
        assert abs(lhs - rhs) < 1e-11 * abs(lhs)
    plan.close()


# Lane-team cases (every FFT size 32 or 64), where the double-float product
# exists: ragged rows (N not a multiple of the team width), unequal axes.
DF_CASES = [c for c in CASES if c[0] in ("woodpile_15", "ellipsoid_21", "woodpile_31", "random_15_21_31",
                                         "random_21_15_15")]


@pytest.mark.parametrize("name,st,n_harm,eps_b,points", DF_CASES, ids=[c[0] for c in DF_CASES])
def test_double_float_apply_matches_oracle(name, st, n_harm, eps_b, points):
    # the arithmetic of the outer residual: pairs of FP32 values with ~48
    # significand bits; an FFT of 64^3 points in it keeps the product within
    # ~1e-13 of the FP64 oracle (the bound asserted leaves a factor ~10)
    g = gsm()
    x = wl.random_field(n_harm, 300 + len(name), batch=len(points))
    plan = g.plan_for(st, n_harm, eps_b=eps_b, precision=g.FP32_REFINE)
    ydf = plan.apply(points, x, precision=g.DF64)
    y64 = plan.apply(points, x, precision=g.FP64)
    for b, pt in enumerate(points):
        want = _oracle_apply(st, n_harm, eps_b, pt, x[b], False)
        assert rel(ydf[b], want) < 1e-12, (name, b, rel(ydf[b], want))
        assert rel(ydf[b], y64[b]) < 1e-12, (name, b, rel(ydf[b], y64[b]))
    plan.close()


def test_double_float_apply_rejects_other_paths():
    g = gsm()
    st = wl.sphere_lattice()
    plan = g.plan_for(st, (7, 7, 7), precision=g.FP32_REFINE)   # FFT size 16: no lane-team product
    x = wl.random_field((7, 7, 7), 5)
    with pytest.raises(g.GsmError) as ei:
        plan.apply([wl.point(0.8 * K0)], x[None], precision=g.DF64)
    assert ei.value.status == g.GSM_ERR_ARG
    plan.close()
    plan = g.plan_for(wl.woodpile(), (15, 15, 15), precision=g.FP32_REFINE)
    x = wl.random_field((15, 15, 15), 6)
    with pytest.raises(g.GsmError) as ei:
        plan.apply([wl.point(0.8 * K0)], x[None], precision=g.DF64, adjoint=True)
    assert ei.value.status == g.GSM_ERR_ARG
    plan.close()
