"""The two complex64 yz passes of the lane-team product (64-point y and z
transforms, two x frequencies per block): team-buffer transposes
(GSM_YZ=smem) and lane-shuffle transposes with phase-deferred spectra
(GSM_YZ=rot).  Both must give the oracle's Eq. 4 operator and the same
refined solutions."""
import numpy as np
import pytest

from oracle import operator as oop
from paper_1501_01752_b300 import workloads as wl

from gpu_common import K0, gsm, oracle_structure, rel

pytestmark = pytest.mark.gpu

CASES = [
    ("woodpile_31", wl.woodpile(), (31, 31, 31),
     [wl.point(0.8 * K0), wl.point(0.7 * K0, (0, 0, 1), (0, 1, 0)), wl.point(0.77 * K0, (0.2, 0.3, 0.9), (1, 0, 0.1))]),
    ("ellipsoid_21", wl.ellipsoid_lattice(), (21, 21, 21), [wl.point(0.83 * K0)]),
    ("random_17_25_29", wl.random_shapes(6, period=(0.3, 0.31, 0.33)), (17, 25, 29),
     [wl.point(0.79 * K0, (0.3, -0.4, 0.8), (0.5, 0.2j, 0.1))]),
]


@pytest.mark.parametrize("variant", ["smem", "rot"])
@pytest.mark.parametrize("name,st,n_harm,points", CASES, ids=[c[0] for c in CASES])
def test_yz_variant_product_matches_oracle(name, st, n_harm, points, variant, monkeypatch):
    monkeypatch.setenv("GSM_YZ", variant)
    g = gsm()
    x = wl.random_field(n_harm, 300 + len(name), batch=len(points))
    plan = g.plan_for(st, n_harm, precision=g.FP64)
    y32 = plan.apply(points, x, precision=g.FP32_REFINE)
    ost = oracle_structure(st)
    Delta = ost.delta(n_harm, 1.0)
    for b, pt in enumerate(points):
        kinc = pt["kappa"] * np.asarray(pt["kdir"])
        want = oop.Operator(Delta, n_harm, kinc, st["periods"], pt["k0"] ** 2)(x[b])
        assert rel(y32[b], want) < 1e-5, (name, variant, b, rel(y32[b], want))
    plan.close()


def test_yz_variants_agree_and_solve_alike(monkeypatch):
    g = gsm()
    st = wl.woodpile()
    n_harm = (31, 31, 31)
    pts = wl.woodpile_batch(16)
    x = wl.random_field(n_harm, 41, batch=4)
    out = {}
    for variant in ("smem", "rot"):
        monkeypatch.setenv("GSM_YZ", variant)
        plan = g.plan_for(st, n_harm, precision=g.FP32_REFINE, tol=1e-8, max_batch=16)
        y = plan.apply(pts[:4], x, precision=g.FP32_REFINE)
        E, infos, s = plan.solve(pts)
        assert s == 0 and all(i["rel_residual"] <= 1e-8 for i in infos)
        out[variant] = (y, E, [i["iters"] for i in infos])
        plan.close()
    # the same product up to complex64 rounding, the same solutions to the refinement tolerance
    assert rel(out["rot"][0], out["smem"][0]) < 2e-6
    assert rel(out["rot"][1], out["smem"][1]) < 1e-7
    assert abs(np.mean(out["rot"][2]) - np.mean(out["smem"][2])) <= 1.0
    ost = oracle_structure(st)
    Delta = ost.delta(n_harm, 1.0)
    E = out["rot"][1].reshape(len(pts), -1)
    for b in (0, 7, 15):
        p = pts[b]
        kinc = p["kappa"] * np.asarray(p["kdir"])
        A = oop.Operator(Delta, n_harm, kinc, st["periods"], p["k0"] ** 2)
        bvec = oop.incident(p["pol"], n_harm)
        res = np.linalg.norm(bvec - A(E[b].reshape((3,) + n_harm[::-1]))) / np.linalg.norm(bvec)
        assert res <= 1.5e-8, (b, res)
