"""Adjoint of the Eq. 4 solve and gradients with respect to the permittivity
(oracle, FP64).  The paper has no adjoint; this is the plain calculus of the
Eq. 4 system, used to check the CUDA adjoint.

With A = I - G T(Delta) and xi = a~^H E (a~ = a at m = 0, zero elsewhere):
    dE  = A^-1 G dT E,
    dxi = lambda^H G dT E,           A^H lambda = a~,
    d xi / d Delta_d = C_d = sum_{m - m' = d} sum_c conj(mu_{c m}) E_{c m'},
    mu  = G^H lambda.
For a voxel cell, Delta_d = (sum_v eps_v phi_v(d) - eps_b delta_d0) / eps_b,
so d xi / d eps_v = sum_d C_d phi_v(d) / eps_b.  For a real objective with
complex gradient g = dL/dRe xi + i dL/dIm xi, dL/d eps_v = Re(conj(g) dxi/deps_v).
"""
from __future__ import annotations

import numpy as np

from . import operator as op
from . import poles
from . import retrieval as rt
from . import solvers


def adjoint_solve(A_op, a, n_harm, tol=1e-12, restart=60, max_iter=5000):
    """lambda with A^H lambda = a~ (GMRES on the adjoint operator)."""
    rhs = op.incident(a, n_harm)
    return solvers.gmres(A_op.adjoint, rhs, tol=tol, restart=restart, max_iter=max_iter)


def coefficient_gradient(A_op, E, lam, n_harm):
    """C_d for d in [-2n, 2n]^3, indexed [dz+2nz, dy+2ny, dx+2nx], by the
    explicit double sum over harmonic pairs (small boxes)."""
    n = op.half(n_harm)
    mu = op.green_apply(np.conj(np.swapaxes(A_op.G, -1, -2)), lam)
    C = np.zeros((4 * n[2] + 1, 4 * n[1] + 1, 4 * n[0] + 1), complex)
    Nz, Ny, Nx = n_harm[2], n_harm[1], n_harm[0]
    for iz in range(Nz):
        for iy in range(Ny):
            for ix in range(Nx):
                # all m' at once: d = m - m'
                block = np.einsum("c,czyx->zyx", np.conj(mu[:, iz, iy, ix]), E)
                C[iz + 2 * n[2] - (Nz - 1):iz + 2 * n[2] + 1,
                  iy + 2 * n[1] - (Ny - 1):iy + 2 * n[1] + 1,
                  ix + 2 * n[0] - (Nx - 1):ix + 2 * n[0] + 1] += block[::-1, ::-1, ::-1]
    return C


def voxel_gradient_from_coeff(C, eps_b, M):
    """d xi / d eps_v = sum_d C_d phi_v(d) / eps_b for an M_z x M_y x M_x grid
    (phi as in coefficients.voxel_coefficients)."""
    D = tuple(s // 2 for s in C.shape)  # (Dz, Dy, Dx)

    def phi(dm, Mm):
        d = np.arange(-dm, dm + 1)[:, None]
        v = np.arange(Mm)[None, :]
        return np.exp(-2j * np.pi * d * (v + 0.5) / Mm) * np.sinc(d / Mm) / Mm

    Mz, My, Mx = M
    pz, py, px = phi(D[0], Mz), phi(D[1], My), phi(D[2], Mx)
    t = np.einsum("cba,av->cbv", C, px)
    t = np.einsum("cbv,bu->cuv", t, py)
    return np.einsum("cuv,cw->wuv", t, pz) / eps_b


def xi_voxel_gradient(structure, n_harm, eps_b, k0, kdir, kappa, a, tol=1e-12):
    """(xi, d xi / d eps_v) for one incident point on a voxel structure."""
    Delta = structure.delta(n_harm, eps_b)
    kinc = kappa * np.asarray(kdir, float) / np.linalg.norm(kdir)
    A = op.Operator(Delta, n_harm, kinc, structure.periods, k0 * k0 * eps_b)
    E, _ = solvers.gmres(A, op.incident(a, n_harm), tol=tol)
    lam, _ = adjoint_solve(A, a, n_harm, tol=tol)
    C = coefficient_gradient(A, E, lam, n_harm)
    return rt.response(E, a, n_harm), voxel_gradient_from_coeff(C, eps_b, structure.voxels.shape)


def component_gradient(structure, n_harm, eps_b, k0, kdir, a, kappas, Np=5, Nd=10, tol=1e-12):
    """(eps_aa, d Re eps_aa / d eps_v) through sweep, pole fit and adjoints."""
    xis, grads = [], []
    for kappa in kappas:
        xi, g = xi_voxel_gradient(structure, n_harm, eps_b, k0, kdir, kappa, a, tol)
        xis.append(xi)
        grads.append(g)
    xis = np.array(xis)
    eta, zeta = poles.fit_poles(kappas, xis, Np, Nd)
    j = poles.select_pole(eta, zeta, kappas.min(), kappas.max())
    d_re, d_im = poles.pole_gradient(kappas, xis, Np, Nd, j)
    deps_deta = 2.0 * eta[j] / k0**2
    out = np.zeros(structure.voxels.shape)
    for i in range(len(kappas)):
        # d Re eps / d Re xi_i and d Re eps / d Im xi_i, combined into g_i
        g = (deps_deta * d_re[i]).real + 1j * (deps_deta * d_im[i]).real
        out += (np.conj(g) * grads[i]).real
    return (eta[j] / k0) ** 2, out
