"""Response sweeps and effective-tensor retrieval (oracle, FP64).

xi(kappa) is the 0th-order response of the "Modes in 3D crystals" section:
the solution of Eq. 4 for the plane-wave source a at |k_inc| = kappa, read as
the projection xi = a^H E_0 on the incident polarisation (reading: the paper
speaks of "0th order vector component amplitude").  Its poles are the mode
propagation constants; with principal axes along x, y, z (the paper's
orthorhombic and tetragonal examples) the propagation constant eta of the
mode travelling along k_dir with field along a gives eps_aa = (eta / k0)^2.
"""
from __future__ import annotations

import numpy as np

from . import coefficients as co
from . import operator as op
from . import poles
from . import solvers


def maxwell_garnett(eps_incl, eps_host, f):
    """Maxwell-Garnett permittivity of spheres at volume fraction f:
    eps_h (1 + 2 f beta) / (1 - f beta), beta = (eps_i - eps_h)/(eps_i + 2 eps_h)
    (the quasistatic comparison of the numerical-convergence section)."""
    beta = (eps_incl - eps_host) / (eps_incl + 2.0 * eps_host)
    return eps_host * (1.0 + 2.0 * f * beta) / (1.0 - f * beta)


class Structure:
    """eps(r) of one cell: host + shapes, or a voxel grid (absolute values)."""

    def __init__(self, periods, eps_host=1.0, shapes=(), voxels=None):
        self.periods = tuple(float(p) for p in periods)
        self.eps_host = eps_host
        self.shapes = list(shapes)
        self.voxels = voxels
        if voxels is not None and self.shapes:
            raise ValueError("give shapes or a voxel grid, not both")

    def eps_coefficients(self, dmax):
        if self.voxels is not None:
            return co.voxel_coefficients(self.voxels, dmax)
        return co.shapes_coefficients(self.eps_host, self.shapes, self.periods, dmax)

    def delta(self, n_harm, eps_b):
        n = op.half(n_harm)
        return co.delta_coefficients(self.eps_coefficients(tuple(2 * a for a in n)), eps_b)

    def inv_eps_coefficients(self, dmax):
        """Fourier coefficients of 1/eps(r), analytic like those of eps."""
        if self.voxels is not None:
            return co.voxel_coefficients(1.0 / np.asarray(self.voxels, complex), dmax)
        inv = [(kind, c, size, 1.0 / complex(eps)) for kind, c, size, eps in self.shapes]
        return co.shapes_coefficients(1.0 / complex(self.eps_host), inv, self.periods, dmax)

    def delta_h(self, n_harm, eps_b):
        """(eps_b/eps - 1)_d, the Toeplitz generator of Eq. 5."""
        n = op.half(n_harm)
        return co.inverse_delta_coefficients(self.inv_eps_coefficients(tuple(2 * a for a in n)), eps_b)


def solve_point(structure, n_harm, eps_b, k0, kdir, kappa, a, method="gmres",
                tol=1e-12, restart=60, max_iter=5000, Delta=None, form="E"):
    """Solve Eq. 4 (form "E": a is the incident E amplitude) or Eq. 5 (form
    "H": a is the incident H amplitude) for one point; returns (field, info)."""
    if Delta is None:
        Delta = structure.delta(n_harm, eps_b) if form == "E" else structure.delta_h(n_harm, eps_b)
    kinc = kappa * np.asarray(kdir, float) / np.linalg.norm(kdir)
    kb2 = k0 * k0 * eps_b
    b = op.incident(a, n_harm)
    if method == "lu":
        dense = op.dense_operator if form == "E" else op.dense_operator_h
        A = dense(Delta, n_harm, kinc, structure.periods, kb2)
        E = solvers.lu_solve(A, b.ravel()).reshape(b.shape)
        return E, dict(iters=0, converged=True)
    Op = op.Operator if form == "E" else op.OperatorH
    A = Op(Delta, n_harm, kinc, structure.periods, kb2, mode="direct" if method == "gmres-direct" else "fft")
    if method == "bicgstab":
        return solvers.bicgstab(A, b, tol=tol, max_iter=max_iter)
    return solvers.gmres(A, b, tol=tol, restart=restart, max_iter=max_iter)


def zeroth_order(E, n_harm):
    """E_0: the three components of the m = 0 harmonic."""
    n = op.half(n_harm)
    return E[:, n[2], n[1], n[0]]


def response(E, a, n_harm):
    """xi = a^H E_0."""
    return np.vdot(np.asarray(a, complex), zeroth_order(E, n_harm))


def kappa_grid(k0, n_centre, rel=0.15, M=16):
    """M equidistant kappa over k0 n_centre [1 - rel, 1 + rel]."""
    return k0 * n_centre * (1.0 + rel * np.linspace(-1.0, 1.0, M))


def sweep(structure, n_harm, eps_b, k0, kdir, a, kappas, method="gmres", tol=1e-12, form="E"):
    Delta = structure.delta(n_harm, eps_b) if form == "E" else structure.delta_h(n_harm, eps_b)
    xs = []
    for kappa in kappas:
        E, _ = solve_point(structure, n_harm, eps_b, k0, kdir, kappa, a, method, tol,
                           Delta=Delta, form=form)
        xs.append(response(E, a, n_harm))
    return np.array(xs)


# (k_dir, a) pairs that excite the principal permittivities eps_xx, eps_yy, eps_zz
PRINCIPAL = ((np.array([0.0, 0.0, 1.0]), np.array([1.0, 0.0, 0.0])),
             (np.array([0.0, 0.0, 1.0]), np.array([0.0, 1.0, 0.0])),
             (np.array([1.0, 0.0, 0.0]), np.array([0.0, 0.0, 1.0])))
# the same modes by their H polarisation (H along k x E): E along x with k
# along z has H along y, E along y has H along x, E along z with k along x
# has H along y
PRINCIPAL_H = ((np.array([0.0, 0.0, 1.0]), np.array([0.0, 1.0, 0.0])),
               (np.array([0.0, 0.0, 1.0]), np.array([1.0, 0.0, 0.0])),
               (np.array([1.0, 0.0, 0.0]), np.array([0.0, 1.0, 0.0])))


def retrieve_component(structure, n_harm, eps_b, k0, kdir, a, kappas, Np=5, Nd=10,
                       method="gmres", tol=1e-12, form="E"):
    """eps_aa = (eta / k0)^2 from the mode pole of xi over the kappa grid."""
    xi = sweep(structure, n_harm, eps_b, k0, kdir, a, kappas, method, tol, form)
    eta, zeta = poles.fit_poles(kappas, xi, Np, Nd)
    j = poles.select_pole(eta, zeta, kappas.min(), kappas.max())
    return (eta[j] / k0) ** 2, dict(eta=eta, zeta=zeta, index=j, xi=xi)


def retrieve_tensor(structure, n_harm, eps_b, k0, kappa_windows, Np=5, Nd=10,
                    method="gmres", tol=1e-12, form="E"):
    """(eps_xx, eps_yy, eps_zz) from the three principal sweeps; kappa_windows
    is a sequence of three kappa grids."""
    out = []
    for (kdir, a), kappas in zip(PRINCIPAL if form == "E" else PRINCIPAL_H, kappa_windows):
        e, _ = retrieve_component(structure, n_harm, eps_b, k0, kdir, a,
                                  np.asarray(kappas, float), Np, Nd, method, tol, form)
        out.append(e)
    return np.array(out)
