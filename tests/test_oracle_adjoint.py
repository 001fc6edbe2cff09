"""Pins for oracle.adjoint: gradients of xi and of the retrieved eps_aa by
central finite differences of the forward oracle."""
import numpy as np

from oracle import adjoint as adj
from oracle import operator as op
from oracle import retrieval as rt
from oracle import solvers
from paper_1501_01752_b300 import workloads as wl

K0 = 2 * np.pi


def _xi_from_delta(Delta, n_harm, kinc, periods, a):
    A = op.dense_operator(Delta, n_harm, kinc, periods, K0**2)
    E = solvers.lu_solve(A, op.incident(a, n_harm).ravel()).reshape((3,) + n_harm[::-1])
    return rt.response(E, a, n_harm)


def test_coefficient_gradient_matches_finite_differences():
    w = wl.random_shapes(8)
    st = rt.Structure(w["periods"], w["eps_host"], w["shapes"])
    n_harm = (3, 3, 5)
    Delta = st.delta(n_harm, 1.0)
    kinc = np.array([0.0, 0.0, 0.85 * K0])
    a = (1.0, 0.0, 0.0)
    A = op.Operator(Delta, n_harm, kinc, w["periods"], K0**2, mode="direct")
    E, _ = solvers.gmres(A, op.incident(a, n_harm), tol=1e-13)
    lam, _ = adj.adjoint_solve(A, a, n_harm, tol=1e-13)
    C = adj.coefficient_gradient(A, E, lam, n_harm)
    h = 1e-6
    for idx in [(4, 2, 2), (0, 0, 0), (7, 3, 1), (2, 4, 3)]:
        Dp, Dm = Delta.copy(), Delta.copy()
        Dp[idx] += h
        Dm[idx] -= h
        fd = (_xi_from_delta(Dp, n_harm, kinc, w["periods"], a)
              - _xi_from_delta(Dm, n_harm, kinc, w["periods"], a)) / (2 * h)
        assert abs(fd - C[idx]) < 1e-6 * max(1.0, abs(C[idx])), (idx, fd, C[idx])


def test_voxel_gradient_matches_finite_differences():
    rng = np.random.default_rng(3)
    vox = np.where(rng.random((6, 5, 4)) > 0.6, 6.0, 1.0)
    st = rt.Structure((0.3, 0.3, 0.3), voxels=vox)
    n_harm = (3, 3, 3)
    args = (st, n_harm, 1.0, K0, (0, 0, 1), 0.9 * K0, (1, 0, 0))
    xi, g = adj.xi_voxel_gradient(*args, tol=1e-13)
    h = 1e-4
    for v in [(0, 0, 0), (5, 4, 3), (2, 1, 3)]:
        vp, vm = vox.copy(), vox.copy()
        vp[v] += h
        vm[v] -= h
        xp = adj.xi_voxel_gradient(rt.Structure((0.3, 0.3, 0.3), voxels=vp), *args[1:], tol=1e-13)[0]
        xm = adj.xi_voxel_gradient(rt.Structure((0.3, 0.3, 0.3), voxels=vm), *args[1:], tol=1e-13)[0]
        fd = (xp - xm) / (2 * h)
        assert abs(fd - g[v]) < 1e-7 * max(1e-3, abs(g[v])), (v, fd, g[v])


def test_retrieved_component_gradient_matches_finite_differences():
    rng = np.random.default_rng(4)
    vox = np.where(rng.random((4, 4, 4)) > 0.7, 4.0, 1.0)
    periods = (0.2, 0.2, 0.2)
    n_harm = (3, 3, 3)
    st = rt.Structure(periods, voxels=vox)
    f = float(np.mean(vox > 2))
    n0 = np.sqrt(rt.maxwell_garnett(4.0, 1.0, f))
    kap = rt.kappa_grid(K0, n0, 0.15, 16)
    eps, g = adj.component_gradient(st, n_harm, 1.0, K0, (0, 0, 1), (1, 0, 0), kap)
    h = 1e-3
    for v in [(0, 0, 0), (3, 2, 1), (1, 3, 2)]:
        vals = []
        for s in (+1, -1):
            vv = vox.copy()
            vv[v] += s * h
            e, _ = rt.retrieve_component(rt.Structure(periods, voxels=vv), n_harm, 1.0, K0,
                                         (0, 0, 1), (1, 0, 0), kap)
            vals.append(e.real)
        fd = (vals[0] - vals[1]) / (2 * h)
        assert abs(fd - g[v]) < 1e-5 * max(1e-3, abs(g[v])), (v, fd, g[v])
