r"""Fourier images of the permittivity of one unit cell (oracle, FP64).

The GSM of the paper never samples eps(r) on a mesh: it uses analytic Fourier
images of simple shapes combined by superposition (GSM section, text after
Eq. 5; "Calculation details", first paragraph).  Convention (the paper leaves
it implicit):

    eps(r) = sum_m eps_m exp(i K_m . r),   K_m = (m_x K_x, m_y K_y, m_z K_z),
    eps_m  = V^-1 \int_cell eps(r) exp(-i K_m . r) d^3r,   K_a = 2 pi / Lambda_a.

A structure is a host permittivity plus non-overlapping shapes, each with its
own permittivity; a shape centred at c contributes
(eps_s - eps_host) exp(-i K_m . c) chi_s(K_m).  Alternatively the cell is a
grid of constant-permittivity voxels, whose coefficients are exact integrals
(not samples) of the piecewise-constant field.

The coefficient that enters Eq. 4 is (Delta eps / eps_b)_d =
(eps_d - eps_b delta_d0) / eps_b.
"""
from __future__ import annotations

import numpy as np

SPHERE, BOX, ELLIPSOID = 0, 1, 2


def _ball_factor(x):
    """3 (sin x - x cos x) / x^3, the normalised Fourier image of a ball of
    unit radius evaluated at |G| R = x.  At x -> 0 the Taylor series
    1 - x^2/10 + x^4/280 replaces the cancelling closed form."""
    x = np.asarray(x, dtype=np.float64)
    out = np.empty_like(x)
    small = np.abs(x) < 1e-2
    xs = x[small]
    out[small] = 1.0 - xs**2 / 10.0 + xs**4 / 280.0
    xl = x[~small]
    out[~small] = 3.0 * (np.sin(xl) - xl * np.cos(xl)) / xl**3
    return out


def shape_image(kind, size, Gx, Gy, Gz, volume):
    """Normalised Fourier image chi(G) = V^-1 \\int_shape exp(-i G.r) d^3r of a
    shape centred at the origin ("Calculation details": analytic images of
    simple shapes).

    kind SPHERE:    size[0] = radius R; f * 3(sin x - x cos x)/x^3, x = |G| R.
    kind BOX:       size = full side lengths; f * prod_a sinc(G_a s_a / 2).
    kind ELLIPSOID: size = semi-axes (a, b, c); the ball image at
                    x = sqrt((G_x a)^2 + (G_y b)^2 + (G_z c)^2).
    f is the shape's volume over the cell volume.
    """
    Gx, Gy, Gz = np.broadcast_arrays(np.asarray(Gx, float), np.asarray(Gy, float),
                                     np.asarray(Gz, float))
    if kind == SPHERE:
        R = float(size[0])
        f = 4.0 * np.pi * R**3 / (3.0 * volume)
        return f * _ball_factor(np.sqrt(Gx**2 + Gy**2 + Gz**2) * R)
    if kind == BOX:
        sx, sy, sz = (float(s) for s in size)
        f = sx * sy * sz / volume
        # np.sinc(u) = sin(pi u)/(pi u), so sinc(G s / 2) = np.sinc(G s / (2 pi))
        return f * (np.sinc(Gx * sx / (2 * np.pi)) * np.sinc(Gy * sy / (2 * np.pi))
                    * np.sinc(Gz * sz / (2 * np.pi)))
    if kind == ELLIPSOID:
        a, b, c = (float(s) for s in size)
        f = 4.0 * np.pi * a * b * c / (3.0 * volume)
        return f * _ball_factor(np.sqrt((Gx * a)**2 + (Gy * b)**2 + (Gz * c)**2))
    raise ValueError(f"unknown shape kind {kind}")


def coefficient_grid(dmax, periods):
    """Integer offsets d in [-dmax_a, dmax_a] per axis and the reciprocal
    vectors G_d = d * K, as broadcastable (z, y, x) arrays."""
    dz = np.arange(-dmax[2], dmax[2] + 1)[:, None, None]
    dy = np.arange(-dmax[1], dmax[1] + 1)[None, :, None]
    dx = np.arange(-dmax[0], dmax[0] + 1)[None, None, :]
    K = [2.0 * np.pi / p for p in periods]
    return (dx, dy, dz), (dx * K[0], dy * K[1], dz * K[2])


def shapes_coefficients(eps_host, shapes, periods, dmax):
    """eps_d for a host permittivity plus non-overlapping shapes.

    shapes: iterable of (kind, center[3], size[3], eps) with eps complex.
    Returns a complex array indexed [dz + dmax_z, dy + dmax_y, dx + dmax_x].
    """
    volume = float(np.prod(periods))
    (dx, dy, dz), (Gx, Gy, Gz) = coefficient_grid(dmax, periods)
    out = np.zeros((2 * dmax[2] + 1, 2 * dmax[1] + 1, 2 * dmax[0] + 1), complex)
    out[dmax[2], dmax[1], dmax[0]] += complex(eps_host)
    for kind, center, size, eps in shapes:
        phase = np.exp(-1j * (Gx * center[0] + Gy * center[1] + Gz * center[2]))
        out += (complex(eps) - complex(eps_host)) * phase * shape_image(kind, size, Gx, Gy, Gz, volume)
    return out


def voxel_coefficients(eps_voxels, dmax):
    """Exact eps_d of a piecewise-constant cell of M_z x M_y x M_x voxels.

    Voxel v = (v_x, v_y, v_z) fills [v_a, v_a + 1) * Lambda_a / M_a along each
    axis, so its integral factorises into one 1D factor per axis:
        phi_a(d, v) = M_a^-1 exp(-2 pi i d (v + 1/2) / M_a) sinc(pi d / M_a)
    and eps_d = sum_v eps_v prod_a phi_a(d_a, v_a).  The sum is written as
    three successive einsum contractions (distributivity only).
    eps_voxels is indexed [v_z, v_y, v_x].
    """
    ev = np.asarray(eps_voxels)
    Mz, My, Mx = ev.shape

    def phi(dm, M):
        d = np.arange(-dm, dm + 1)[:, None]
        v = np.arange(M)[None, :]
        return np.exp(-2j * np.pi * d * (v + 0.5) / M) * np.sinc(d / M) / M

    px, py, pz = phi(dmax[0], Mx), phi(dmax[1], My), phi(dmax[2], Mz)
    t = np.einsum("zyx,ax->zya", ev.astype(complex), px)
    t = np.einsum("zya,by->zba", t, py)
    return np.einsum("zba,cz->cba", t, pz)


def delta_coefficients(eps_d, eps_b):
    """(Delta eps / eps_b)_d = (eps_d - eps_b delta_d0) / eps_b, the Toeplitz
    generator of Eq. 4."""
    out = np.array(eps_d, dtype=complex, copy=True)
    c = tuple(s // 2 for s in out.shape)
    out[c] -= eps_b
    return out / eps_b


def inverse_delta_coefficients(inv_eps_d, eps_b):
    """[delta - eps_b/eps]_d with the sign of Eq. 5 folded into its use: this
    returns (eps_b/eps - 1)_d = eps_b (1/eps)_d - delta_d0, the Toeplitz
    generator of the H-field formulation.  inv_eps_d are the Fourier
    coefficients of 1/eps(r), found analytically like those of eps
    ("Calculation details": no numerical inversion of the eps matrix)."""
    out = eps_b * np.array(inv_eps_d, dtype=complex, copy=True)
    c = tuple(s // 2 for s in out.shape)
    out[c] -= 1.0
    return out
