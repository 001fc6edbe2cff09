"""Pins of the oracle's H-field formulation (Eq. 5) against closed forms,
invariants of the operator and the E-field formulation (Eq. 4)."""
import numpy as np
import pytest

from oracle import operator as op
from oracle import retrieval as rt
from paper_1501_01752_b300 import workloads as wl

from test_oracle_physics import K0, _bloch_in_plane, _bloch_normal, _stack


def test_homogeneous_medium_closed_form_h():
    # eps(r) = eps1 everywhere: (eps_b/eps - 1)_d = (eps_b/eps1 - 1) delta_d0 and
    # k x (k x h) = -kappa^2 h for transverse h, so the m = 0 block alone gives
    # H_0 = h (kappa^2 - k_b^2) / (kappa^2 eps_b/eps1 - k_b^2); a longitudinal h
    # is left unchanged (k x h = 0); every other harmonic vanishes.
    eps1, eps_b = 2.25, 1.3
    st = rt.Structure((0.3, 0.31, 0.32), eps_host=eps1)
    n_harm = (3, 5, 3)
    kb2 = K0**2 * eps_b
    for kappa in (0.7 * K0, 1.21 * K0, 1.9 * K0):
        for method in ("lu", "gmres"):
            H, _ = rt.solve_point(st, n_harm, eps_b, K0, (0, 0, 1), kappa, (0.6, 0.8, 0), method=method, form="H")
            H0 = rt.zeroth_order(H, n_harm)
            want = np.array([0.6, 0.8, 0]) * (kappa**2 - kb2) / (kappa**2 * eps_b / eps1 - kb2)
            assert np.allclose(H0, want, atol=1e-12)
            assert abs(np.linalg.norm(H) - np.linalg.norm(H0)) < 1e-12
        H, _ = rt.solve_point(st, n_harm, eps_b, K0, (0, 0, 1), kappa, (0, 0, 1.0), method="lu", form="H")
        assert np.allclose(rt.zeroth_order(H, n_harm), [0, 0, 1.0], atol=1e-12)


def test_homogeneous_pole_and_residue_h():
    # xi(kappa) = (kappa^2 - k_b^2) eps1 / (eps_b (kappa^2 - eta^2)): the pole is
    # the exact dispersion eta = k0 sqrt(eps1), the residue eps1 (eta^2 - k_b^2) / (2 eta eps_b)
    eps1, eps_b = 2.25, 1.0
    st = rt.Structure((0.3, 0.3, 0.3), eps_host=eps1)
    kap = rt.kappa_grid(K0, 1.5, 0.15, 16)
    eps, d = rt.retrieve_component(st, (3, 3, 3), eps_b, K0, (0, 0, 1), (0, 1, 0), kap, form="H")
    eta = d["eta"][d["index"]]
    assert abs(eps - eps1) < 1e-9
    assert abs(d["zeta"][d["index"]] - eps1 * (eta**2 - K0**2) / (2 * eta * eps_b)) < 1e-7


def _random_case():
    w = wl.random_shapes(3)
    st = rt.Structure(w["periods"], w["eps_host"], w["shapes"])
    n_harm = (5, 3, 5)
    k = np.array([0.3, 0.5, 0.8])
    kinc = 0.9 * K0 * k / np.linalg.norm(k)
    return st, n_harm, kinc


def test_fft_form_equals_explicit_matrix_h():
    st, n_harm, kinc = _random_case()
    Dh = st.delta_h(n_harm, 1.0)
    A = op.dense_operator_h(Dh, n_harm, kinc, st.periods, K0**2)
    Af = op.OperatorH(Dh, n_harm, kinc, st.periods, K0**2)
    Ad = op.OperatorH(Dh, n_harm, kinc, st.periods, K0**2, mode="direct")
    rng = np.random.default_rng(3)
    x = rng.standard_normal(A.shape[0]) + 1j * rng.standard_normal(A.shape[0])
    want = A @ x
    assert np.linalg.norm(Af(x).ravel() - want) < 1e-13 * np.linalg.norm(want)
    assert np.linalg.norm(Ad(x).ravel() - want) < 1e-13 * np.linalg.norm(want)


def test_operator_structure_h():
    # diag(k^2 - k_b^2) A_H = diag(k^2 - k_b^2) - [k x] T [k x] is Hermitian for
    # real eps and real k ([k x] is real antisymmetric, the Toeplitz matrix of
    # a real function Hermitian): a transposed Toeplitz or a dropped sign in a
    # cross product breaks it on this non-centrosymmetric cell.
    st, n_harm, kinc = _random_case()
    A = op.dense_operator_h(st.delta_h(n_harm, 1.0), n_harm, kinc, st.periods, K0**2)
    kf = op.wavevector_field(n_harm, kinc, st.periods)
    den = np.tile((kf * kf).sum(-1).ravel() - K0**2, 3)
    M = den[:, None] * A
    assert np.abs(M - M.conj().T).max() < 1e-13 * np.abs(M).max()


def test_solution_is_transverse_and_response_real_h():
    # the longitudinal part of H never couples (k x h_L = 0), so a transverse
    # source gives k_m . H_m = 0 at every harmonic; the Hermitian structure
    # above makes h^T H_0 real for real h (lossless medium)
    st, n_harm, kinc = _random_case()
    kappa = np.linalg.norm(kinc)
    h = np.cross(kinc, [1, 0, 0])
    h /= np.linalg.norm(h)
    H, _ = rt.solve_point(st, n_harm, 1.0, K0, kinc / kappa, kappa, h, method="lu", form="H")
    kf = op.wavevector_field(n_harm, kinc, st.periods)
    div = np.einsum("zyxa,azyx->zyx", kf, H)
    assert np.abs(div).max() < 1e-13 * np.abs(kf).max() * np.abs(H).max()
    xi = h @ rt.zeroth_order(H, n_harm)
    assert abs(xi.imag) < 1e-12 * abs(xi)


def test_layered_stack_h_converges_to_bloch():
    # Laurent truncation of 1/eps: the field tangential to the layers (normal
    # incidence) converges ~1/N here (fast in the E-form); E normal to the
    # layers (in-plane TM) is much closer than in the E-form at equal N
    st = _stack()
    for n_ref, kdir, h, bound in ((_bloch_normal() / K0, (0, 0, 1), (0, 1, 0), 1e-2),
                                  (_bloch_in_plane(True) / K0, (1, 0, 0), (0, 1, 0), 5e-4)):
        errs = []
        for Nz in (21, 41):
            kap = rt.kappa_grid(K0, n_ref, 0.15, 16)
            eps, _ = rt.retrieve_component(st, (1, 1, Nz), 1.0, K0, kdir, h, kap, form="H")
            errs.append(abs(np.sqrt(eps).real - n_ref))
        assert errs[1] < bound and 0.4 < errs[1] / errs[0] < 0.6, (n_ref, errs)


def test_e_and_h_forms_bracket_and_approach_each_other():
    # sphere lattice: the E-form estimate of eps_xx lies above the H-form one
    # and the gap shrinks as the truncation grows (both tend to the same mode)
    s = wl.sphere_lattice()
    st = rt.Structure(s["periods"], s["eps_host"], s["shapes"])
    n0 = np.sqrt(rt.maxwell_garnett(4.0, 1.0, 4 * np.pi * 0.3**3 / 3))
    kap = rt.kappa_grid(K0, n0, 0.15, 16)
    gaps = []
    for N in (5, 7, 9):
        eE, _ = rt.retrieve_component(st, (N,) * 3, 1.0, K0, (0, 0, 1), (1, 0, 0), kap, form="E")
        eH, _ = rt.retrieve_component(st, (N,) * 3, 1.0, K0, (0, 0, 1), (0, 1, 0), kap, form="H")
        assert eE.real > eH.real
        gaps.append(eE.real - eH.real)
    assert gaps[2] < gaps[1] < gaps[0] and gaps[2] < 0.6 * gaps[0]


def _dense_h_mutant(Delta_h, n_harm, kinc, periods, kb2, mutation):
    # the oracle's Eq. 5 matrix with one plausible mistake planted
    T = op.toeplitz_matrix(Delta_h, n_harm)
    k = op.wavevector_field(n_harm, kinc, periods).reshape(-1, 3)
    Nh = T.shape[0]
    den = (k * k).sum(-1) - kb2
    if mutation == "denominator_sign":
        den = -den
    Cx = np.zeros((3 * Nh, 3 * Nh))
    for a in range(3):
        b, c = (a + 1) % 3, (a + 2) % 3
        Cx[a * Nh:(a + 1) * Nh, c * Nh:(c + 1) * Nh] += np.diag(k[:, b])
        Cx[a * Nh:(a + 1) * Nh, b * Nh:(b + 1) * Nh] -= np.diag(k[:, c])
    TT = np.kron(np.eye(3), T)
    right = -Cx if mutation == "swapped_cross" else Cx     # H x k instead of k x H
    return np.eye(3 * Nh) - np.tile(1.0 / den, 3)[:, None] * (Cx @ TT @ right)


@pytest.mark.parametrize("mutation", ["denominator_sign", "swapped_cross", "multiplier_sign"])
def test_h_mutations_fail_a_pin(mutation):
    # each mistake specific to Eq. 5 breaks the homogeneous closed form or the
    # Hermitian structure (the pins above).  The Toeplitz orientation is the
    # builder shared with Eq. 4 and pinned there (a transposed Toeplitz of a
    # real eps is its complex conjugate, the mirrored cell, which is still
    # Hermitian).
    eps1 = 2.25
    hom = rt.Structure((0.3, 0.3, 0.3), eps_host=eps1)
    n_harm = (3, 3, 3)
    kappa = 1.2 * K0
    kinc = np.array([0.0, 0.0, kappa])
    Dh = hom.delta_h(n_harm, 1.0)
    if mutation == "multiplier_sign":
        Dh = -Dh                                            # (1 - eps_b/eps) instead of (eps_b/eps - 1)
    b = op.incident((0, 1, 0), n_harm).ravel()
    H0 = np.linalg.solve(_dense_h_mutant(Dh, n_harm, kinc, hom.periods, K0**2, mutation), b)
    want = (kappa**2 - K0**2) / (kappa**2 / eps1 - K0**2)
    closed_form_ok = abs(H0.reshape(3, 3, 3, 3)[1, 1, 1, 1] - want) < 1e-9
    st, nh, ki = _random_case()
    A = _dense_h_mutant(st.delta_h(nh, 1.0), nh, ki, st.periods, K0**2, mutation)
    kf = op.wavevector_field(nh, ki, st.periods)
    den = np.tile((kf * kf).sum(-1).ravel() - K0**2, 3)
    M = den[:, None] * A
    hermitian_ok = np.abs(M - M.conj().T).max() < 1e-13 * np.abs(M).max()
    assert not (closed_form_ok and hermitian_ok), mutation
