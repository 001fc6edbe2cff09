"""The right preconditioner of the GMRES solves (averaged-medium block
diagonal of Eq. 4, GSM_PRECOND_AUTO): it must leave every solution as the
oracle computes it (FP64 to 1e-10, complex64 + refinement to 1e-6), cut the
number of products on a high-contrast lattice, and fall back to a smaller
scale where a point sits on the light cone of the averaged medium."""
import numpy as np
import pytest

from oracle import retrieval as ort
from paper_1501_01752_b300 import workloads as wl

from gpu_common import K0, gsm, oracle_structure, rel

pytestmark = pytest.mark.gpu

N15 = (15, 15, 15)   # 32-point lane-team grid


def _oracle(st, n_harm, pt, tol=1e-12):
    E, info = ort.solve_point(oracle_structure(st), n_harm, 1.0, pt["k0"], pt["kdir"], pt["kappa"], pt["pol"],
                              method="gmres", tol=tol)
    assert info["converged"]
    return E.ravel()


def _points():
    pts = wl.woodpile_batch(6)
    pts.append(wl.point(0.75 * K0, (0.6, 0.0, 0.8), (0.0, 1.0, 0.0)))
    # just above the light cone of the averaged medium (eps 3.725 for the
    # woodpile): the m = 0 harmonic makes M = I - Delta_0 G singular at s = 1
    pts.append(wl.point(np.sqrt(3.725) * 1.001 * K0, (0.0, 0.0, 1.0), (1.0, 0.0, 0.0)))
    return pts


def _split(E, n):
    return E.reshape(n, -1)


@pytest.mark.parametrize("prec", ["refine", "fp64"])
def test_preconditioned_solves_match_oracle(prec):
    g = gsm()
    st = wl.woodpile()
    pts = _points()
    kw = dict(precision=g.FP32_REFINE, tol=1e-8) if prec == "refine" else dict(precision=g.FP64, tol=1e-12)
    res = {}
    for pc in (g.PRECOND_AUTO, g.PRECOND_NONE):
        plan = g.plan_for(st, N15, max_batch=len(pts), precond=pc, **kw)
        E, infos, s = plan.solve(pts)
        assert s == 0, infos
        res[pc] = (_split(E, len(pts)), infos)
        plan.close()
    bound = 1e-6 if prec == "refine" else 1e-10
    for b in (0, 3, 6, 7):
        want = _oracle(st, N15, pts[b])
        for pc in res:
            assert rel(res[pc][0][b], want) < bound, (pc, b, rel(res[pc][0][b], want))
    for b in range(len(pts)):
        assert rel(res[g.PRECOND_AUTO][0][b], res[g.PRECOND_NONE][0][b]) < 2 * bound
    it_pc = sum(i["iters"] for i in res[g.PRECOND_AUTO][1][:6])
    it_no = sum(i["iters"] for i in res[g.PRECOND_NONE][1][:6])
    assert it_pc < 0.9 * it_no, (it_pc, it_no)


def test_preconditioned_31_harmonics_refined_residuals():
    """The bench truncation (31^3 on the 64^3 grid): every returned field
    satisfies Eq. 4 to 1e-8 by the oracle's own FFT operator."""
    from oracle import operator as oop
    g = gsm()
    st = wl.woodpile()
    n_harm = (31, 31, 31)
    pts = wl.woodpile_batch(4)
    plan = g.plan_for(st, n_harm, precision=g.FP32_REFINE, tol=1e-8, max_batch=4)
    E, infos, s = plan.solve(pts)
    assert s == 0
    plan.close()
    ost = oracle_structure(st)
    Delta = ost.delta(n_harm, 1.0)
    for b, pt in enumerate(pts):
        kinc = pt["kappa"] * np.asarray(pt["kdir"])
        A = oop.Operator(Delta, n_harm, kinc, st["periods"], pt["k0"] ** 2)
        rhs = oop.incident(pt["pol"], n_harm)
        r = rhs - A(_split(E, 4)[b].reshape(A.shape))
        assert np.linalg.norm(r) / np.linalg.norm(rhs) < 1.2e-8


def test_preconditioned_128_point_teams_gyroid():
    """The 128-point lane-team path (33 harmonics per axis on the 128^3 grid)
    with the preconditioner (gyroid voxels, eps 12, Delta_0 = 3.7): refined
    solves satisfy Eq. 4 to 1e-8 by the oracle's own FFT operator, agree with
    the unpreconditioned solves, and take fewer products."""
    from oracle import operator as oop
    g = gsm()
    vox = wl.gyroid_voxels(32, 0.5, (1.0, 12.0))
    st = dict(periods=(0.4, 0.4, 0.4), voxels=vox)
    n_harm = (33, 33, 33)
    pts = [wl.point(0.8 * K0), wl.point(0.85 * K0, (0.0, 0.6, 0.8), (1.0, 0.0, 0.0))]
    res = {}
    for pc in (g.PRECOND_AUTO, g.PRECOND_NONE):
        plan = g.plan_for(st, n_harm, precision=g.FP32_REFINE, tol=1e-8, max_batch=2, precond=pc)
        assert plan.level_fft() == (128, 128, 128)
        E, infos, s = plan.solve(pts)
        assert s == 0, infos
        res[pc] = (_split(E, 2), sum(i["iters"] for i in infos))
        plan.close()
    Delta = oracle_structure(st).delta(n_harm, 1.0)
    for b, pt in enumerate(pts):
        kinc = pt["kappa"] * np.asarray(pt["kdir"]) / np.linalg.norm(pt["kdir"])
        A = oop.Operator(Delta, n_harm, kinc, st["periods"], pt["k0"] ** 2)
        rhs = oop.incident(pt["pol"], n_harm)
        r = rhs - A(res[g.PRECOND_AUTO][0][b].reshape(A.shape))
        assert np.linalg.norm(r) / np.linalg.norm(rhs) < 1.2e-8
        assert rel(res[g.PRECOND_AUTO][0][b], res[g.PRECOND_NONE][0][b]) < 2e-6
    assert res[g.PRECOND_AUTO][1] < res[g.PRECOND_NONE][1], (res[g.PRECOND_AUTO][1], res[g.PRECOND_NONE][1])


@pytest.mark.parametrize("n_harm", [N15, (31, 31, 31)])
def test_preconditioned_operator_matches_oracle(n_harm):
    # gsm_apply op 2 (the product the solves iterate with) against the
    # oracle's Eq. 4 operator applied to M^{-1} x, M = I - Delta_0 G(m)
    # inverted here as an explicit 3 x 3 matrix per harmonic; the points are
    # chosen where the largest scale s = 1 qualifies (checked below)
    from oracle import operator as oop
    g = gsm()
    st = wl.woodpile()
    ost = oracle_structure(st)
    Delta = ost.delta(n_harm, 1.0)
    d0 = Delta[tuple(s // 2 for s in Delta.shape)].real
    pts = [wl.point(0.8 * K0), wl.point(0.72 * K0, (0, 0, 1), (0, 1, 0)),
           wl.point(0.75 * K0, (0.6, 0.0, 0.8), (0.0, 1.0, 0.0))]
    x = wl.random_field(n_harm, 77, batch=len(pts))
    plan = g.plan_for(st, n_harm, precision=g.FP64)
    y64 = plan.apply(pts, x, precision=g.FP64, precond=True)
    y32 = plan.apply(pts, x, precision=g.FP32_REFINE, precond=True)
    for b, pt in enumerate(pts):
        kinc = pt["kappa"] * np.asarray(pt["kdir"])
        kb2 = pt["k0"] ** 2
        kx, ky, kz = oop.wavevectors(n_harm, kinc, st["periods"])
        KZ, KY, KX = np.meshgrid(kz, ky, kx, indexing="ij")
        k2 = KX ** 2 + KY ** 2 + KZ ** 2
        assert np.min(np.abs(k2 - kb2 * (1 + d0))) >= 0.1 * abs(d0) * kb2   # s = 1 qualifies
        G = oop.green(n_harm, kinc, st["periods"], kb2)
        Minv = np.linalg.inv(np.eye(3) - d0 * G)
        u = np.einsum("zyxab,bzyx->azyx", Minv, x[b])
        want = oop.Operator(Delta, n_harm, kinc, st["periods"], kb2)(u)
        assert rel(y64[b], want) < 1e-12, (b, rel(y64[b], want))
        assert rel(y32[b], want) < 1e-5, (b, rel(y32[b], want))
    plan.close()
