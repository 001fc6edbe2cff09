"""Linear solvers for Eq. 4 (oracle, FP64).

The paper solves the truncated Eq. 4 by GMRES in Saad's formulation with
modified Gram-Schmidt orthogonalisation ("Calculation details", program
paragraph), and names BiCGSTAB as the alternative that fails near poles (GSM
section, truncation paragraph; "Calculation details").  Dense LU with partial
pivoting is the plain definition of the solution for small boxes.

Readings where the paper is silent: x0 = 0; the tolerance is on
||b - A x|| / ||b||; full GMRES up to ``restart`` Arnoldi steps, then restart
from the current iterate; complex Givens rotations; no preconditioner.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg


def lu_solve(A, b):
    """Dense LU with partial pivoting (LAPACK getrf/getrs via scipy)."""
    lu, piv = scipy.linalg.lu_factor(A)
    return scipy.linalg.lu_solve((lu, piv), b)


def _dot(u, v):
    return np.vdot(u, v)  # conj(u) . v


def gmres(apply, b, tol=1e-10, restart=60, max_iter=2000, x0=None):
    """GMRES(m) with modified Gram-Schmidt Arnoldi and Givens rotations.

    Returns (x, info) with info = dict(iters, rel_residual, history, converged)
    where history holds the Givens residual estimate after every Arnoldi step
    and rel_residual is the true ||b - A x|| / ||b|| at exit.
    """
    b = np.asarray(b, complex)
    shape = b.shape
    b = b.ravel()
    x = np.zeros_like(b) if x0 is None else np.asarray(x0, complex).ravel().copy()
    bnorm = np.linalg.norm(b)
    if bnorm == 0.0:
        return x.reshape(shape), dict(iters=0, rel_residual=0.0, history=[], converged=True)
    A = lambda v: np.asarray(apply(v.reshape(shape))).ravel()
    iters, history = 0, []
    while True:
        r = b - A(x) if iters or x0 is not None else b.copy()
        beta = np.linalg.norm(r)
        if beta / bnorm <= tol or iters >= max_iter:
            break
        m = restart
        V = [r / beta]
        H = np.zeros((m + 1, m), complex)
        cs = np.zeros(m)
        sn = np.zeros(m, complex)
        g = np.zeros(m + 1, complex)
        g[0] = beta
        k = 0
        for j in range(m):
            w = A(V[j])
            iters += 1
            for i in range(j + 1):                      # modified Gram-Schmidt
                H[i, j] = _dot(V[i], w)
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            for i in range(j):                          # previous rotations
                hi, hi1 = H[i, j], H[i + 1, j]
                H[i, j] = cs[i] * hi + sn[i] * hi1
                H[i + 1, j] = -np.conj(sn[i]) * hi + cs[i] * hi1
            a, bb = H[j, j], H[j + 1, j]
            rho = np.hypot(abs(a), abs(bb))
            if abs(a) == 0.0:
                cs[j], sn[j] = 0.0, 1.0
            else:
                cs[j] = abs(a) / rho
                sn[j] = (a / abs(a)) * np.conj(bb) / rho
            H[j, j] = cs[j] * a + sn[j] * bb
            H[j + 1, j] = 0.0
            g[j + 1] = -np.conj(sn[j]) * g[j]
            g[j] = cs[j] * g[j]
            k = j + 1
            history.append(abs(g[j + 1]) / bnorm)
            hnext = np.linalg.norm(w)
            if history[-1] <= tol or iters >= max_iter or hnext == 0.0:
                break
            V.append(w / hnext)
        y = scipy.linalg.solve_triangular(H[:k, :k], g[:k])
        for i in range(k):
            x = x + y[i] * V[i]
    rel = np.linalg.norm(b - A(x)) / bnorm
    return x.reshape(shape), dict(iters=iters, rel_residual=rel, history=history,
                                  converged=bool(rel <= tol))


def bicgstab(apply, b, tol=1e-10, max_iter=2000):
    """BiCGSTAB (van der Vorst) with shadow residual r_hat = r_0 and x0 = 0."""
    b = np.asarray(b, complex)
    shape = b.shape
    b = b.ravel()
    A = lambda v: np.asarray(apply(v.reshape(shape))).ravel()
    bnorm = np.linalg.norm(b)
    x = np.zeros_like(b)
    r = b.copy()
    rhat = r.copy()
    rho_old = alpha = omega = 1.0 + 0j
    v = np.zeros_like(b)
    p = np.zeros_like(b)
    it = 0
    history = []
    while it < max_iter:
        rho = _dot(rhat, r)
        if rho == 0:
            break
        beta = (rho / rho_old) * (alpha / omega)
        p = r + beta * (p - omega * v)
        v = A(p)
        alpha = rho / _dot(rhat, v)
        s = r - alpha * v
        t = A(s)
        tt = _dot(t, t)
        omega = _dot(t, s) / tt if tt != 0 else 0.0
        x = x + alpha * p + omega * s
        r = s - omega * t
        rho_old = rho
        it += 1
        history.append(np.linalg.norm(r) / bnorm)
        if history[-1] <= tol or omega == 0:
            break
    rel = np.linalg.norm(b - A(x)) / bnorm
    return x.reshape(shape), dict(iters=it, rel_residual=rel, history=history,
                                  converged=bool(rel <= tol))


def minres(apply_h, c, precond=None, tol=1e-10, max_iter=2000):
    """Preconditioned MINRES (Paige and Saunders) for a Hermitian, possibly
    indefinite H: minimises ||c - H x|| in the norm of precond^{-1} over the
    Krylov space of precond^{-1} H, with a three-term Lanczos recurrence (real
    coefficients for Hermitian H) and Givens rotations.  precond(r) applies
    M^{-1} of a Hermitian positive definite M (None = identity).  Stops when
    the recurrence's residual estimate phibar falls to tol * beta1.

    Used for the Hermitian form of the lossless Eq. 4 (G^{-1} - Delta) E =
    G^{-1} E_inc, a Krylov variant the paper does not use; returns (x, info)
    as gmres does, with iters = products with H."""
    c = np.asarray(c, complex)
    shape = c.shape
    c = c.ravel()
    H = lambda v: np.asarray(apply_h(v.reshape(shape))).ravel()
    Mi = (lambda v: v) if precond is None else (lambda v: np.asarray(precond(v.reshape(shape))).ravel())
    x = np.zeros_like(c)
    r1 = c.copy()
    y = Mi(r1)
    beta1 = np.sqrt(np.vdot(r1, y).real)
    if beta1 == 0.0:
        return x.reshape(shape), dict(iters=0, history=[], converged=True)
    oldb, beta, dbar, epsln, phibar = 0.0, beta1, 0.0, 0.0, beta1
    cs, sn = -1.0, 0.0
    w = np.zeros_like(c)
    w2 = np.zeros_like(c)
    r2 = r1.copy()
    history = []
    it = 0
    while it < max_iter:
        v = y / beta
        y = H(v)
        it += 1
        if it >= 2:
            y = y - (beta / oldb) * r1
        alfa = np.vdot(v, y).real
        y = y - (alfa / beta) * r2
        r1, r2 = r2, y
        y = Mi(r2)
        oldb, beta = beta, np.sqrt(max(np.vdot(r2, y).real, 0.0))
        oldeps = epsln
        delta = cs * dbar + sn * alfa
        gbar = sn * dbar - cs * alfa
        epsln = sn * beta
        dbar = -cs * beta
        gamma = max(np.hypot(gbar, beta), np.finfo(float).tiny)
        cs, sn = gbar / gamma, beta / gamma
        phi = cs * phibar
        phibar = sn * phibar
        w1, w2 = w2, w
        w = (v - oldeps * w1 - delta * w2) / gamma
        x = x + phi * w
        history.append(abs(phibar) / beta1)
        if history[-1] <= tol or beta == 0.0:
            break
    return x.reshape(shape), dict(iters=it, history=history, converged=bool(history and history[-1] <= tol))
