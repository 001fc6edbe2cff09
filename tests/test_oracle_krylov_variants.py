"""Krylov variants of the lossless Eq. 4 on the oracle (CPU, FP64).

The paper solves Eq. 4 by GMRES and names BiCGSTAB as an alternative that
fails near poles ("Calculation details", GSM truncation paragraph).  For
real eps and real k the system has the Hermitian form (G^{-1} - Delta) E =
G^{-1} E_inc, which MINRES can use.  These tests pin the oracle's MINRES and
record the comparison that kept it out of the CUDA path: it needs more
products than GMRES or BiCGSTAB for the same Eq. 4 residual."""
import numpy as np
import pytest

from oracle import operator as oop
from oracle import retrieval as ort
from oracle import solvers as osv
from paper_1501_01752_b300 import workloads as wl

K0 = 2 * np.pi


def test_minres_matches_dense_solve_on_hermitian_indefinite_systems():
    rng = np.random.default_rng(11)
    n = 80
    B = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    H = B + B.conj().T                                  # Hermitian, indefinite
    assert np.min(np.linalg.eigvalsh(H)) < 0 < np.max(np.linalg.eigvalsh(H))
    c = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    want = np.linalg.solve(H, c)
    d = rng.uniform(0.5, 3.0, n)                        # Hermitian positive definite preconditioner
    for pre in (None, lambda r: r / d):
        x, info = osv.minres(lambda v: H @ v, c, precond=pre, tol=1e-13, max_iter=1000)
        assert info["converged"]
        assert np.linalg.norm(x - want) / np.linalg.norm(want) < 1e-10


def test_minres_terminates_after_as_many_steps_as_distinct_eigenvalues():
    # a Hermitian matrix with 5 distinct eigenvalues (both signs): the
    # Krylov space is exhausted after 5 products
    rng = np.random.default_rng(12)
    Q, _ = np.linalg.qr(rng.standard_normal((40, 40)) + 1j * rng.standard_normal((40, 40)))
    lam = np.repeat([-3.0, -1.0, 0.5, 2.0, 7.0], 8)
    H = (Q * lam) @ Q.conj().T
    c = rng.standard_normal(40) + 0j
    x, info = osv.minres(lambda v: H @ v, c, tol=1e-12, max_iter=40)
    assert info["iters"] == 5
    assert np.linalg.norm(H @ x - c) / np.linalg.norm(c) < 1e-11


def _hermitian_form(st, n_harm, kappa, kdir=(0, 0, 1)):
    """Eq. 4's operator A, the Hermitian H = G^{-1} - Delta with H E = G^{-1} b,
    and the positive definite preconditioner |G^{-1}|^{-1} per harmonic."""
    ost = ort.Structure(st["periods"], st["eps_host"], st["shapes"])
    Delta = ost.delta(n_harm, 1.0)
    kinc = kappa * np.asarray(kdir, float) / np.linalg.norm(kdir)
    A = oop.Operator(Delta, n_harm, kinc, st["periods"], K0 ** 2)
    Gi = np.linalg.inv(oop.green(n_harm, kinc, st["periods"], K0 ** 2))
    w, U = np.linalg.eigh(Gi)
    Pinv = np.einsum("...ij,...j,...kj->...ik", U, 1.0 / np.abs(w), U.conj())
    shape = (3,) + tuple(n_harm[::-1])
    app = lambda M, v: np.einsum("zyxab,bzyx->azyx", M, v.reshape(shape))
    H = lambda v: app(Gi, v) - A.toeplitz(v.reshape(shape))
    return A, H, (lambda r: app(Pinv, r)), Gi, app, Delta


def test_hermitian_form_is_hermitian_and_gives_the_eq4_solution():
    st = wl.random_shapes(7)
    n_harm = (5, 5, 5)
    A, H, pre, Gi, app, Delta = _hermitian_form(st, n_harm, 0.77 * K0, (0.3, -0.2, 0.9))
    U = 3 * 125
    Hd = np.stack([np.asarray(H(e)).ravel() for e in np.eye(U)], axis=1)
    assert np.abs(Hd - Hd.conj().T).max() < 1e-12 * np.abs(Hd).max()
    b = oop.incident((0.2, 0.5, 0.1j), n_harm)
    kinc = 0.77 * K0 * np.array([0.3, -0.2, 0.9]) / np.linalg.norm([0.3, -0.2, 0.9])
    want = osv.lu_solve(oop.dense_operator(Delta, n_harm, kinc, st["periods"], K0 ** 2), b.ravel())
    x, info = osv.minres(H, app(Gi, b), precond=pre, tol=1e-13, max_iter=2000)
    assert np.linalg.norm(x.ravel() - want) / np.linalg.norm(want) < 1e-9


@pytest.mark.parametrize("kappa", [0.8, 0.72])
def test_krylov_products_on_the_woodpile(kappa):
    # products to ||b - A E|| <= 1e-8 ||b|| on the woodpile at 15^3 harmonics
    # (plain operator, no averaged-medium preconditioner): GMRES 40-41,
    # BiCGSTAB 56-58, MINRES on the Hermitian form with the |G^{-1}|
    # preconditioner 76.  MINRES stops on its own preconditioned residual
    # estimate, so its tolerance is tightened until the Eq. 4 residual meets
    # the target.
    st = wl.woodpile()
    n_harm = (15, 15, 15)
    A, H, pre, Gi, app, _ = _hermitian_form(st, n_harm, kappa * K0)
    b = oop.incident((1, 0, 0), n_harm)
    bn = np.linalg.norm(b)
    xg, ig = osv.gmres(A, b, tol=1e-8, restart=60)
    xb, ib = osv.bicgstab(A, b, tol=1e-8)
    assert ig["converged"] and ib["converged"]
    for mt in (1e-8, 1e-9, 1e-10, 1e-11):
        xm, im = osv.minres(H, app(Gi, b), precond=pre, tol=mt, max_iter=3000)
        rm = np.linalg.norm(b - A(xm)) / bn
        if rm <= 1e-8:
            break
    assert rm <= 1e-8
    n_gmres, n_bicg, n_minres = ig["iters"], 2 * ib["iters"], im["iters"]
    assert 35 <= n_gmres <= 45 and 50 <= n_bicg <= 64 and 70 <= n_minres <= 82, (n_gmres, n_bicg, n_minres)
    assert n_minres > n_bicg > n_gmres
    # the three agree on the solution
    for x in (xb, xm):
        assert np.linalg.norm(x - xg) / np.linalg.norm(xg) < 1e-6
