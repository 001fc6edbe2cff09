"""BiCGSTAB (the Krylov method the paper names beside GMRES) in the CUDA
path: batched, inside the same refinement loop, checked against the oracle's
dense LU / GMRES solutions and the oracle's own residual of the returned
fields."""
import numpy as np
import pytest

from oracle import adjoint as oadj
from oracle import operator as oop
from oracle import retrieval as ort
from paper_1501_01752_b300 import workloads as wl

from gpu_common import K0, gsm, oracle_structure, rel

pytestmark = pytest.mark.gpu


def _fields(plan, pts, E):
    out, off = [], 0
    for p in pts:
        n = plan.field_size(p)
        out.append(E[off:off + n])
        off += n
    return out


def _oracle(st, n_harm, pt, method="lu", tol=1e-13):
    E, _ = ort.solve_point(oracle_structure(st), n_harm, 1.0, pt["k0"], pt["kdir"], pt["kappa"], pt["pol"],
                           method=method, tol=tol)
    return E.ravel()


def _oracle_residual(st, n_harm, pt, E):
    Delta = oracle_structure(st).delta(n_harm, 1.0)
    A = oop.Operator(Delta, n_harm, pt["kappa"] * np.asarray(pt["kdir"]), st["periods"], pt["k0"] ** 2)
    b = oop.incident(pt["pol"], n_harm)
    return float(np.linalg.norm(b - A(E.reshape(b.shape))) / np.linalg.norm(b))


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_bicgstab_matches_dense_lu(prec):
    g = gsm()
    st = wl.sphere_lattice()
    n_harm = (7, 7, 7)
    pts = [wl.point(0.8 * K0), wl.point(0.8 * K0, (0, 0, 1), (0, 1, 0)), wl.point(0.6 * K0, (1, 1, 0), (0, 0, 1)),
           wl.point(1.05 * K0, (0, 0, 1), (1, 0, 0))]
    fp64 = prec == "fp64"
    plan = g.plan_for(st, n_harm, precision=g.FP64 if fp64 else g.FP32_REFINE, tol=1e-12 if fp64 else 1e-8,
                      krylov=g.BICGSTAB)
    E, infos, s = plan.solve(pts)
    assert s == 0
    for b, (p, Eb) in enumerate(zip(pts, _fields(plan, pts, E))):
        want = _oracle(st, n_harm, p)
        assert infos[b]["rel_residual"] <= (1e-12 if fp64 else 1e-8), infos[b]
        assert rel(Eb, want) < (1e-10 if fp64 else 1e-6), (b, rel(Eb, want))
        assert infos[b]["iters"] >= 2
    plan.close()


def test_bicgstab_woodpile_31_refined():
    g = gsm()
    st = wl.woodpile()
    n_harm = (31, 31, 31)
    pts = wl.woodpile_batch(4)
    plan = g.plan_for(st, n_harm, precision=g.FP32_REFINE, tol=1e-8, krylov=g.BICGSTAB)
    E, infos, s = plan.solve(pts)
    assert s == 0
    for b, (p, Eb) in enumerate(zip(pts, _fields(plan, pts, E))):
        assert _oracle_residual(st, n_harm, p, Eb) <= 1.5e-8, (b, infos[b])
        if b < 2:
            want = _oracle(st, n_harm, p, method="gmres", tol=1e-12)
            assert rel(Eb, want) < 1e-6, (b, rel(Eb, want))
    plan.close()


def test_bicgstab_mixed_truncations_and_graph_free_path(monkeypatch):
    g = gsm()
    st = wl.ellipsoid_lattice()
    pts = []
    for i, N in enumerate([(5, 5, 5), (9, 9, 9), (5, 5, 5), (7, 9, 5), (9, 9, 9)]):
        p = wl.point((0.7 + 0.05 * i) * K0, (0, 0, 1), (1, 0, 0) if i % 2 == 0 else (0, 1, 0))
        p["n_harm"] = N
        pts.append(p)
    plan = g.plan_for(st, (9, 9, 9), precision=g.FP64, tol=1e-12, max_batch=2, krylov=g.BICGSTAB)
    E, infos, s = plan.solve(pts)
    plan.close()
    assert s == 0
    for p, Eb in zip(pts, _fields(plan, pts, E)):
        assert rel(Eb, _oracle(st, p["n_harm"], p)) < 1e-10
    # the iterations launched one by one (no CUDA graph) run the same kernels
    monkeypatch.setenv("GSM_GRAPHS", "0")
    plan = g.plan_for(st, (9, 9, 9), precision=g.FP64, tol=1e-12, max_batch=2, krylov=g.BICGSTAB)
    E2, infos2, s2 = plan.solve(pts)
    plan.close()
    assert s2 == 0 and rel(E2, E) < 1e-13
    assert [i["iters"] for i in infos2] == [i["iters"] for i in infos]


def test_bicgstab_memory_cap_and_iteration_limit():
    g = gsm()
    st = wl.woodpile()
    n_harm = (15, 15, 15)
    U = 3 * 15 ** 3
    pt = wl.point(0.8 * K0)
    # seven complex64 vectors per instance fit in this cap; GMRES would restart every 6 steps
    plan = g.plan_for(st, n_harm, precision=g.FP32_REFINE, tol=1e-8, hbm_cap=7 * U * 8, max_batch=1,
                      krylov=g.BICGSTAB)
    E, infos, s = plan.solve([pt])
    assert s == 0 and infos[0]["rel_residual"] <= 1e-8
    assert rel(E, _oracle(st, n_harm, pt, method="gmres", tol=1e-12)) < 1e-6
    plan.close()
    plan = g.plan_for(st, n_harm, precision=g.FP32_REFINE, tol=1e-8, hbm_cap=6 * U * 8, max_batch=1,
                      krylov=g.BICGSTAB)
    with pytest.raises(g.GsmError) as ei:
        plan.solve([pt])
    assert ei.value.status == g.GSM_ERR_NOMEM
    plan.close()
    plan = g.plan_for(st, (7, 7, 7), precision=g.FP64, tol=1e-14, max_iter=4, krylov=g.BICGSTAB)
    E, infos, s = plan.solve([pt])
    assert s == g.GSM_ERR_NOCONV and infos[0]["status"] == g.GSM_ERR_NOCONV
    assert np.all(np.isfinite(E)) and infos[0]["rel_residual"] < 1.0
    plan.close()


def test_bicgstab_adjoint_gradient_matches_oracle():
    # the adjoint solve A^H lambda = g by BiCGSTAB, then the same gradient
    g = gsm()
    rng = np.random.default_rng(7)
    vox = np.where(rng.random((8, 8, 8)) < 0.3, 6.0, 1.0)
    periods = (0.3, 0.3, 0.3)
    n_harm = (5, 5, 5)
    st = dict(periods=periods, voxels=vox)
    pts = [wl.point(0.9 * K0), wl.point(0.95 * K0, (0, 0, 1), (0, 1, 0))]
    plan = g.plan_for(st, n_harm, precision=g.FP64, tol=1e-13, krylov=g.BICGSTAB)
    cs = [1.0, 0.5 - 0.25j]
    gE0 = np.array([c * np.asarray(p["pol"]) for c, p in zip(cs, pts)])
    got = plan.adjoint(pts, gE0)
    ost = ort.Structure(periods, voxels=vox)
    want = np.zeros_like(vox)
    for c, p in zip(cs, pts):
        _, dxi = oadj.xi_voxel_gradient(ost, n_harm, 1.0, p["k0"], p["kdir"], p["kappa"], p["pol"], tol=1e-13)
        want += (np.conj(c) * dxi).real
    assert rel(got, want) < 1e-8, rel(got, want)
    plan.close()
