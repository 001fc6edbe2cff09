"""The truncated GSM operator of Eq. 4 (oracle, FP64).

Eq. 4 written as a linear system A E = E_inc on the truncated harmonic box
m in [-n_x, n_x] x [-n_y, n_y] x [-n_z, n_z] (N_a = 2 n_a + 1 per axis,
GSM section, truncation paragraph):

    (A E)_{a m} = E_{a m} - sum_b G_{ab}(m) sum_{m'} Delta_{m - m'} E_{b m'},
    G_{ab}(m)   = (k_b^2 delta_ab - k_{a m} k_{b m}) / (k_m^2 - k_b^2),
    k_{a m}     = k^inc_a + m_a K_a,   K_a = 2 pi / Lambda_a,
    Delta_d     = (Delta eps / eps_b)_d,
    E^inc_{a m} = delta_{m 0} a_a                      (plane-wave source).

Field layout: complex array (3, N_z, N_y, N_x), component first, x fastest,
index [c, m_z + n_z, m_y + n_y, m_x + n_x].  Delta is indexed
[d_z + D_z, d_y + D_y, d_x + D_x] with D_a >= 2 n_a.
"""
from __future__ import annotations

import numpy as np
import scipy.fft

# scipy.fft worker threads used by the FFT form of the operator; the CPU
# baseline raises it to the host core count.
WORKERS = 1


def half(n_harm):
    """n_a = (N_a - 1) / 2 for odd N_a (only odd, symmetric boxes exist)."""
    for N in n_harm:
        if N < 1 or N % 2 == 0:
            raise ValueError("harmonic counts must be odd and positive")
    return tuple((N - 1) // 2 for N in n_harm)


def wavevectors(n_harm, kinc, periods):
    """k_{a m} = k^inc_a + m_a K_a for each axis (text after Eq. 4)."""
    n = half(n_harm)
    return tuple(kinc[a] + np.arange(-n[a], n[a] + 1) * (2.0 * np.pi / periods[a])
                 for a in range(3))


def green(n_harm, kinc, periods, kb2):
    """G(m) of Eq. 4 for every harmonic, shape (N_z, N_y, N_x, 3, 3)."""
    kx, ky, kz = wavevectors(n_harm, kinc, periods)
    KZ, KY, KX = np.meshgrid(kz, ky, kx, indexing="ij")
    k = np.stack([KX, KY, KZ], axis=-1)
    k2 = (k * k).sum(-1)
    num = kb2 * np.eye(3) - k[..., :, None] * k[..., None, :]
    den = k2 - kb2
    if np.any(np.abs(den) <= 1e-12 * max(abs(kb2), 1.0)):
        raise ZeroDivisionError("k_m^2 = k_b^2 for some harmonic (Eq. 4 needs k_m^2 != k_b^2)")
    return num / den[..., None, None]


def incident(a, n_harm):
    """E^inc_{a m} = delta_{m0} a_a (plane wave, text after Eq. 4)."""
    n = half(n_harm)
    b = np.zeros((3,) + tuple(n_harm[::-1]), complex)
    b[:, n[2], n[1], n[0]] = np.asarray(a, complex)
    return b


def toeplitz_matrix(Delta, n_harm):
    """T[m, m'] = Delta_{m - m'} over the flattened (z, y, x) harmonic box."""
    n = half(n_harm)
    D = tuple(s // 2 for s in Delta.shape)  # (D_z, D_y, D_x)
    mz, my, mx = np.meshgrid(np.arange(-n[2], n[2] + 1), np.arange(-n[1], n[1] + 1),
                             np.arange(-n[0], n[0] + 1), indexing="ij")
    mz, my, mx = mz.ravel(), my.ravel(), mx.ravel()
    return Delta[(mz[:, None] - mz[None, :]) + D[0],
                 (my[:, None] - my[None, :]) + D[1],
                 (mx[:, None] - mx[None, :]) + D[2]]


def dense_operator(Delta, n_harm, kinc, periods, kb2):
    """The explicit 3N x 3N matrix of Eq. 4, ordering [c][m_z][m_y][m_x]."""
    T = toeplitz_matrix(Delta, n_harm)
    G = green(n_harm, kinc, periods, kb2).reshape(-1, 3, 3)
    Nh = T.shape[0]
    A = np.zeros((3 * Nh, 3 * Nh), complex)
    for a in range(3):
        for b in range(3):
            A[a * Nh:(a + 1) * Nh, b * Nh:(b + 1) * Nh] = -G[:, a, b][:, None] * T
        A[a * Nh:(a + 1) * Nh, a * Nh:(a + 1) * Nh] += np.eye(Nh)
    return A


def toeplitz_apply_direct(Delta, x, n_harm):
    """u_m = sum_{m'} Delta_{m-m'} x_{m'} per component, by the explicit
    Toeplitz matrix (small boxes only)."""
    T = toeplitz_matrix(Delta, n_harm)
    return np.stack([(T @ x[c].ravel()).reshape(x[c].shape) for c in range(3)])


def toeplitz_apply_fft(Delta, x, n_harm):
    """The same product as a cyclic convolution on a grid of L_a = 2 N_a - 1
    points per axis (paper: the Toeplitz product is accelerated by the FFT).

    Every offset d = m - m' in [-2n, 2n] has a distinct residue mod L_a, so the
    cyclic convolution of Delta (placed at d mod L) and x (placed at m mod L)
    equals the truncated Toeplitz product on the box.
    """
    n = half(n_harm)
    L = tuple(2 * N - 1 for N in n_harm)          # (L_x, L_y, L_z)
    shape = (L[2], L[1], L[0])
    D = tuple(s // 2 for s in Delta.shape)
    dz = np.arange(-2 * n[2], 2 * n[2] + 1)
    dy = np.arange(-2 * n[1], 2 * n[1] + 1)
    dx = np.arange(-2 * n[0], 2 * n[0] + 1)
    Dp = np.zeros(shape, complex)
    Dp[np.ix_(dz % L[2], dy % L[1], dx % L[0])] = Delta[np.ix_(dz + D[0], dy + D[1], dx + D[2])]
    FD = scipy.fft.fftn(Dp, workers=WORKERS)
    mz = np.arange(-n[2], n[2] + 1) % L[2]
    my = np.arange(-n[1], n[1] + 1) % L[1]
    mx = np.arange(-n[0], n[0] + 1) % L[0]
    xp = np.zeros((3,) + shape, complex)
    xp[(slice(None),) + np.ix_(mz, my, mx)] = x
    conv = scipy.fft.ifftn(FD[None] * scipy.fft.fftn(xp, axes=(1, 2, 3), workers=WORKERS),
                           axes=(1, 2, 3), workers=WORKERS)
    return conv[(slice(None),) + np.ix_(mz, my, mx)]


def green_apply(G, u):
    """(G u)_{a m} = sum_b G_ab(m) u_{b m}."""
    return np.einsum("zyxab,bzyx->azyx", G, u)


class Operator:
    """y = A x for Eq. 4 with a fixed structure and incident point.

    mode "fft" (any size) or "direct" (explicit Toeplitz matrix, small boxes).
    """

    def __init__(self, Delta, n_harm, kinc, periods, kb2, mode="fft"):
        self.Delta, self.n_harm = Delta, tuple(n_harm)
        self.G = green(n_harm, kinc, periods, kb2)
        self.mode = mode
        self.shape = (3,) + tuple(n_harm[::-1])

    def toeplitz(self, x):
        if self.mode == "direct":
            return toeplitz_apply_direct(self.Delta, x, self.n_harm)
        return toeplitz_apply_fft(self.Delta, x, self.n_harm)

    def __call__(self, x):
        x = np.asarray(x, complex).reshape(self.shape)
        return x - green_apply(self.G, self.toeplitz(x))

    def adjoint(self, v):
        """A^H v = v - T^H (G^H v); T^H is the Toeplitz product with
        conj(Delta_{-d}) (the Hermitian transpose of T[m,m'] = Delta_{m-m'})."""
        v = np.asarray(v, complex).reshape(self.shape)
        Gh = np.conj(np.swapaxes(self.G, -1, -2))
        w = green_apply(Gh, v)
        DeltaH = np.conj(self.Delta[::-1, ::-1, ::-1])
        if self.mode == "direct":
            return v - toeplitz_apply_direct(DeltaH, w, self.n_harm)
        return v - toeplitz_apply_fft(DeltaH, w, self.n_harm)


# --------------------------------------------------------------- Eq. 5
# The H-field formulation (GSM section, Eq. 5):
#
#   H_m = H^inc_m + k_m x [ sum_m' (delta_{mm'} - (eps_b/eps)_{m-m'}) (k_m' x H_m') ] / (k_b^2 - k_m^2),
#
# i.e. with Delta'_d = (eps_b/eps - 1)_d the system A_H H = H^inc,
#
#   (A_H H)_m = H_m - k_m x (Delta' * (k x H))_m / (k_m^2 - k_b^2),
#
# where * is the Toeplitz (truncated convolution) product of every Cartesian
# component.  Re-derived from curl (eps^-1 curl H) = k0^2 H: for a mode
# exp(i k.r) with k.H = 0, curl curl -> k^2, so
# (k_m^2 - k_b^2) H_m = k_m x sum_m' (eps_b/eps - 1)_{m-m'} (k_m' x H_m').

def wavevector_field(n_harm, kinc, periods):
    """k_m for every harmonic, shape (N_z, N_y, N_x, 3)."""
    kx, ky, kz = wavevectors(n_harm, kinc, periods)
    KZ, KY, KX = np.meshgrid(kz, ky, kx, indexing="ij")
    return np.stack([KX, KY, KZ], axis=-1)


def cross_apply(k, v):
    """(k x v)_m for v of shape (3, N_z, N_y, N_x) and k of shape (N_z, N_y, N_x, 3)."""
    kk = np.moveaxis(k, -1, 0)
    return np.cross(kk, v, axis=0)


def dense_operator_h(Delta_h, n_harm, kinc, periods, kb2):
    """The explicit 3N x 3N matrix of Eq. 5, ordering [c][m_z][m_y][m_x]:
    A_H = I - diag(1/(k^2 - k_b^2)) C T C with C = per-harmonic k x, T the
    Toeplitz matrix of Delta' applied to each component."""
    T = toeplitz_matrix(Delta_h, n_harm)
    k = wavevector_field(n_harm, kinc, periods).reshape(-1, 3)
    Nh = T.shape[0]
    den = (k * k).sum(-1) - kb2
    if np.any(np.abs(den) <= 1e-12 * max(abs(kb2), 1.0)):
        raise ZeroDivisionError("k_m^2 = k_b^2 for some harmonic")
    # cross-product matrix [k x] per harmonic: (k x v)_a = eps_abc k_b v_c
    Cx = np.zeros((3 * Nh, 3 * Nh))
    for a in range(3):
        b, c = (a + 1) % 3, (a + 2) % 3
        Cx[a * Nh:(a + 1) * Nh, c * Nh:(c + 1) * Nh] += np.diag(k[:, b])
        Cx[a * Nh:(a + 1) * Nh, b * Nh:(b + 1) * Nh] -= np.diag(k[:, c])
    TT = np.zeros((3 * Nh, 3 * Nh), complex)
    for a in range(3):
        TT[a * Nh:(a + 1) * Nh, a * Nh:(a + 1) * Nh] = T
    Dinv = np.tile(1.0 / den, 3)
    return np.eye(3 * Nh) - Dinv[:, None] * (Cx @ TT @ Cx)


class OperatorH:
    """y = A_H x for Eq. 5 with a fixed structure and incident point (the
    Toeplitz products by FFT, or by the explicit matrix with mode "direct")."""

    def __init__(self, Delta_h, n_harm, kinc, periods, kb2, mode="fft"):
        self.Delta, self.n_harm = Delta_h, tuple(n_harm)
        self.k = wavevector_field(n_harm, kinc, periods)
        den = (self.k * self.k).sum(-1) - kb2
        if np.any(np.abs(den) <= 1e-12 * max(abs(kb2), 1.0)):
            raise ZeroDivisionError("k_m^2 = k_b^2 for some harmonic")
        self.iden = 1.0 / den
        self.mode = mode
        self.shape = (3,) + tuple(n_harm[::-1])

    def toeplitz(self, x):
        if self.mode == "direct":
            return toeplitz_apply_direct(self.Delta, x, self.n_harm)
        return toeplitz_apply_fft(self.Delta, x, self.n_harm)

    def __call__(self, x):
        x = np.asarray(x, complex).reshape(self.shape)
        u = cross_apply(self.k, self.toeplitz(cross_apply(self.k, x)))
        return x - self.iden[None] * u
