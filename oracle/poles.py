"""Resonance model and pole fit of the "Modes in 3D crystals" section
(oracle, FP64): Eq. 6 (meromorphic response), Eq. 7 (pole polynomial),
Eq. 8 (divided-difference annihilation), Eq. 9 (linear system for p_k),
QR eigenvalues of the companion matrix, Eq. 10 (residues).

Readings of passages that are garbled or silent in the text:
  * Eq. 9 as printed carries xi_i in a denominator.  Eq. 8 applies the divided
    difference to P(kappa) xi(kappa), whose divided difference over points
    kappa_0..kappa_Nd is sum_i P(kappa_i) xi_i / prod_{j!=i}(kappa_i - kappa_j);
    xi_i therefore multiplies, and the system used is
      sum_{k<Np} [sum_i kappa_i^k xi_i c_i] p_k = -sum_i kappa_i^Np xi_i c_i,
      c_i = 1 / prod_{j != i} (kappa_i - kappa_j),  p_Np = 1.
  * "N_p - 1 independent point sets" gives one equation fewer than the N_p
    unknowns p_0..p_{Np-1}.  Reading: M >= N_d + N_p equidistant points, every
    window of N_d + 1 consecutive points gives one row (S = M - N_d rows), and
    the rows are solved in the least-squares sense.
  * Eq. 10's upper limit "m" is N_p: zeta_k = (P xi)(eta_k) / P'(eta_k) with
    (P xi)(eta_k) the Lagrange interpolant over one window of N_d + 1 points,
    evaluated at eta_k.  The window used is the one whose centre is nearest
    Re eta_k.
  * kappa is mapped affinely to t = (kappa - c) / h (c, h the centre and
    half-width of the grid) before the divided differences are formed; this
    is exact in exact arithmetic (poles map to c + h tau, residues to
    h zeta_t) and keeps the order-N_d differences representable.
"""
from __future__ import annotations

import numpy as np


def dd_weights(t):
    """c_i = 1 / prod_{j != i} (t_i - t_j): the weights of the Newton divided
    difference of order len(t) - 1 (Eq. 8)."""
    t = np.asarray(t)
    diff = t[:, None] - t[None, :]
    np.fill_diagonal(diff, 1.0)
    return 1.0 / np.prod(diff, axis=1)


def lagrange_basis(t, z):
    """L_i(z) = prod_{j != i} (z - t_j) / (t_i - t_j) for every node t_i."""
    t = np.asarray(t)
    out = np.empty(len(t), complex)
    for i in range(len(t)):
        others = np.delete(t, i)
        out[i] = np.prod((z - others) / (t[i] - others))
    return out


def _normalise(kappa):
    kappa = np.asarray(kappa, float)
    c = 0.5 * (kappa.max() + kappa.min())
    h = 0.5 * (kappa.max() - kappa.min())
    return (kappa - c) / h, c, h


def system_rows(t, xi, Np, Nd):
    """Rows of Eq. 9 (reading above): one row per window of Nd+1 points.
    Returns (R, r) with R of shape (S, Np)."""
    M = len(t)
    S = M - Nd
    R = np.zeros((S, Np), complex)
    r = np.zeros(S, complex)
    for w in range(S):
        tw, xw = t[w:w + Nd + 1], xi[w:w + Nd + 1]
        c = dd_weights(tw)
        for k in range(Np):
            R[w, k] = np.sum(tw**k * xw * c)
        r[w] = -np.sum(tw**Np * xw * c)
    return R, r


def companion_roots(p):
    """Roots of the monic t^Np + sum_{k<Np} p_k t^k as eigenvalues of its
    companion matrix (LAPACK Hessenberg QR via numpy)."""
    Np = len(p)
    C = np.zeros((Np, Np), complex)
    C[1:, :-1] = np.eye(Np - 1)
    C[:, -1] = -np.asarray(p)
    return np.linalg.eigvals(C)


def fit_poles(kappa, xi, Np=5, Nd=10):
    """Poles eta_j and residues zeta_j of xi(kappa) (Eqs. 7-10).

    kappa: M >= Nd + Np equidistant real points; xi: M complex responses.
    Returns (eta, zeta), each of length Np, in kappa units.
    """
    xi = np.asarray(xi, complex)
    M = len(xi)
    if Nd <= Np or M < Nd + Np:
        raise ValueError("need Nd > Np and at least Nd + Np points")
    t, c, h = _normalise(kappa)
    R, r = system_rows(t, xi, Np, Nd)
    p = np.linalg.lstsq(R, r, rcond=None)[0]
    tau = companion_roots(p)
    zeta_t = np.empty(Np, complex)
    centres = np.array([t[w + Nd // 2] for w in range(M - Nd)])
    for k in range(Np):
        w = int(np.argmin(np.abs(centres - tau[k].real)))
        tw, xw = t[w:w + Nd + 1], xi[w:w + Nd + 1]
        P_at_nodes = np.array([np.prod(ti - tau) for ti in tw])
        Pxi = np.sum(P_at_nodes * xw * lagrange_basis(tw, tau[k]))
        dP = np.prod(np.delete(tau[k] - tau, k))
        zeta_t[k] = Pxi / dP
    return c + h * tau, h * zeta_t


def select_pole(eta, zeta, lo, hi):
    """The mode pole: largest |zeta| among poles with lo <= Re eta <= hi
    (reading: the paper picks the propagating mode's pole in the sweep
    interval without stating a rule)."""
    inside = [j for j in range(len(eta)) if lo <= eta[j].real <= hi]
    if not inside:
        raise ValueError("no pole inside the kappa interval")
    return max(inside, key=lambda j: abs(zeta[j]))


def pole_gradient(kappa, xi, Np, Nd, index):
    """d eta_index / d Re(xi_i) and d eta_index / d Im(xi_i) for every i.

    Reading (the paper differentiates nothing): the fitted poles move with
    the data as the poles of the Eq. 6 model.  Linearising it around the
    poles that matter in the window (the selected one and every other fitted
    pole with |Re t| <= 1.5 and a residue above 1e-8 of the largest; at most
    (M - Nd) / 2 of them, nearest first) gives
        d xi(t) = sum_j [d zeta_j/(t - tau_j) + zeta_j d tau_j/(t - tau_j)^2]
                  + d regular(t),
    with the regular part a Chebyshev polynomial of degree Nd - 2 in the
    normalised t.  The least-squares row of d tau_index over the M samples is
    d tau / d xi_i.  (Direct differentiation of the Eq. 9 least-squares
    solution is not used: the order-Nd divided-difference rows have condition
    numbers near 1e14 and lose every digit of dp.)  Pinned against finite
    differences of fit_poles.
    """
    xi = np.asarray(xi, complex)
    eta, zeta = fit_poles(kappa, xi, Np, Nd)
    t, c, h = _normalise(kappa)
    tau = (eta - c) / h
    zt = zeta / h
    big = np.abs(zt) > 1e-8 * np.max(np.abs(zt))
    cand = [j for j in range(len(tau)) if j != index and big[j] and abs(tau[j].real) <= 1.5]
    cand.sort(key=lambda j: abs(tau[j] - tau[index]))
    explicit = [index] + cand[: max(0, (len(t) - Nd) // 2 - 1)]
    cols = []
    for j in explicit:
        cols.append(1.0 / (t - tau[j]))
        cols.append(zt[j] / (t - tau[j]) ** 2)
    for l in range(Nd - 1):
        cols.append(np.cos(l * np.arccos(np.clip(t, -1.0, 1.0))) + 0j)
    J = np.stack(cols, axis=1)
    w = np.linalg.pinv(J)[1] * h
    return w, 1j * w
