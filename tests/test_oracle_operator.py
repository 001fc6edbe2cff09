"""Pins for oracle.operator (Eq. 4) and oracle.solvers."""
import numpy as np

from oracle import operator as op
from oracle import solvers
from oracle import retrieval as rt
from paper_1501_01752_b300 import workloads as wl

K0 = 2 * np.pi


def _rand(rng, shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def test_toeplitz_product_is_fourier_coefficient_of_a_product():
    # eps(r) and E(r) band-limited trigonometric polynomials: the Fourier
    # coefficients of the pointwise product eps(r) E(r), found by explicit DFT
    # sums on a grid fine enough for no aliasing, are exactly
    # sum_m' eps_{m-m'} E_m' (the orientation of the Toeplitz index in Eq. 4).
    rng = np.random.default_rng(5)
    n = (1, 2, 1)
    n_harm = tuple(2 * a + 1 for a in n)
    Delta = _rand(rng, (4 * n[2] + 1, 4 * n[1] + 1, 4 * n[0] + 1))
    x = _rand(rng, (3,) + n_harm[::-1])
    P = [6 * a + 1 for a in n]  # grid points per axis
    g = [np.arange(P[a]) / P[a] for a in range(3)]

    def synth(coef, half):
        # f(r) = sum_m c_m exp(2 pi i m.r), r on the grid
        ms = [np.arange(-half[a], half[a] + 1) for a in range(3)]
        ex = [np.exp(2j * np.pi * np.outer(g[a], ms[a])) for a in range(3)]
        return np.einsum("zyx,Zz,Yy,Xx->ZYX", coef, ex[2], ex[1], ex[0])

    def analyse(f, half):
        ms = [np.arange(-half[a], half[a] + 1) for a in range(3)]
        ex = [np.exp(-2j * np.pi * np.outer(ms[a], g[a])) / P[a] for a in range(3)]
        return np.einsum("ZYX,zZ,yY,xX->zyx", f, ex[2], ex[1], ex[0])

    eps_r = synth(Delta, tuple(2 * a for a in n))
    want = np.stack([analyse(eps_r * synth(x[c], n), n) for c in range(3)])
    got = op.toeplitz_apply_direct(Delta, x, n_harm)
    assert np.max(np.abs(got - want)) < 1e-11 * np.max(np.abs(want))
    got_fft = op.toeplitz_apply_fft(Delta, x, n_harm)
    assert np.max(np.abs(got_fft - want)) < 1e-11 * np.max(np.abs(want))


def test_green_tensor_inverts_the_curl_curl_symbol():
    # Eq. 4 comes from curl curl E - k_b^2 E = k_b^2 Delta E; in Fourier space
    # curl -> i k, so Q(m) v = -k x (k x v) - k_b^2 v and G(m) Q(m) = k_b^2 I.
    n_harm = (3, 5, 3)
    kinc = np.array([0.3, -0.2, 0.9]) * K0
    periods = (0.3, 0.33, 0.36)
    kb2 = K0**2 * 1.7
    G = op.green(n_harm, kinc, periods, kb2)
    kx, ky, kz = op.wavevectors(n_harm, kinc, periods)
    for iz in range(3):
        for iy in range(5):
            for ix in range(3):
                k = np.array([kx[ix], ky[iy], kz[iz]])
                Q = np.stack([-np.cross(k, np.cross(k, e)) - kb2 * e for e in np.eye(3)], axis=1)
                assert np.max(np.abs(G[iz, iy, ix] @ Q - kb2 * np.eye(3))) < 1e-9 * kb2


def test_fft_form_equals_explicit_toeplitz():
    rng = np.random.default_rng(7)
    for n_harm in [(3, 5, 7), (5, 5, 5), (1, 1, 9)]:
        D = tuple(2 * (N - 1) for N in n_harm)  # 4n per axis
        Delta = _rand(rng, (D[2] + 1, D[1] + 1, D[0] + 1))
        x = _rand(rng, (3,) + n_harm[::-1])
        a = op.toeplitz_apply_direct(Delta, x, n_harm)
        b = op.toeplitz_apply_fft(Delta, x, n_harm)
        assert np.max(np.abs(a - b)) < 1e-12 * np.max(np.abs(a))


def test_dense_matrix_equals_operator_and_adjoint_identity():
    rng = np.random.default_rng(11)
    n_harm = (3, 5, 3)
    Delta = _rand(rng, (9, 17, 9)) * 0.3   # lossy, non-Hermitian
    kinc = np.array([0.1, 0.2, 0.7]) * K0
    periods = (0.3, 0.33, 0.36)
    A = op.dense_operator(Delta, n_harm, kinc, periods, K0**2)
    Aop = op.Operator(Delta, n_harm, kinc, periods, K0**2)
    x = _rand(rng, (3,) + n_harm[::-1])
    y = _rand(rng, (3,) + n_harm[::-1])
    assert np.allclose((A @ x.ravel()).reshape(x.shape), Aop(x), atol=1e-12)
    assert np.allclose((A.conj().T @ y.ravel()).reshape(y.shape), Aop.adjoint(y), atol=1e-12)
    assert abs(np.vdot(Aop(x), y) - np.vdot(x, Aop.adjoint(y))) < 1e-10 * np.linalg.norm(x) * np.linalg.norm(y)


def test_gmres_and_bicgstab_match_dense_lu():
    s = wl.sphere_lattice()
    st = rt.Structure(s["periods"], s["eps_host"], s["shapes"])
    n_harm = (7, 7, 7)
    args = (st, n_harm, 1.0, K0, (0, 0, 1), 0.8 * K0, (1, 0, 0))
    E_lu, _ = rt.solve_point(*args, method="lu")
    for method, kw in [("gmres", {}), ("gmres", dict(restart=5)), ("bicgstab", {})]:
        E, info = rt.solve_point(*args, method=method, tol=1e-12, **kw)
        assert info["converged"]
        assert np.linalg.norm(E - E_lu) / np.linalg.norm(E_lu) < 1e-10, method


def test_gmres_exact_on_small_known_system():
    # diagonal system with three distinct eigenvalues: GMRES terminates in 3 steps
    d = np.array([1.0, 2.0, 2.0, 3.0, 1.0 + 1j] * 4)
    b = np.arange(1, 21) + 0j
    x, info = solvers.gmres(lambda v: d * v, b, tol=1e-13)
    assert info["iters"] == 4 and np.allclose(x, b / d, atol=1e-12)


def test_singular_harmonic_is_rejected():
    import pytest
    with pytest.raises(ZeroDivisionError):
        op.green((1, 1, 1), np.array([0, 0, K0]), (0.3, 0.3, 0.3), K0**2)
