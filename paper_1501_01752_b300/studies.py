"""Parameter studies of the paper's effective-anisotropy section (Figs. 4
and 5): lattices of spherical air cavities in a matrix of index 1.5 whose
periods change at a fixed volume filling factor, their principal effective
indices (the retrieval of Eqs. 6-10 through the C ABI), and cross-sections
of the normal surface from mode searches along off-axis directions.

Everything here orchestrates library calls (gsm_retrieve_tensor, gsm_sweep,
gsm_fit_poles); the arithmetic of the solves runs in libgsm.  Fresnel's
equation is the effective-medium reference the off-axis indices are
compared with.

    python -m paper_1501_01752_b300.studies fig4 [--harm 9] [--out fig4.json]
    python -m paper_1501_01752_b300.studies fig5 [--harm 9] [--out fig5.json]
"""
from __future__ import annotations

import argparse
import json
import math

import numpy as np

from . import gsm
from . import workloads as wl

K0 = 2.0 * math.pi        # lengths in vacuum wavelengths
N_HOST = 1.5
RADII = (0.01, 0.02, 0.03, 0.04, 0.05)   # cavity radii of the figures, in wavelengths


def maxwell_garnett(eps_i, eps_h, f):
    """Isotropic Maxwell-Garnett permittivity (the figures' horizontal line)."""
    b = (eps_i - eps_h) / (eps_i + 2.0 * eps_h)
    return eps_h * (1.0 + 2.0 * f * b) / (1.0 - f * b)


def tetragonal_periods(ratio, radius, f=4.0 * math.pi / 81.0):
    """Fig. 4: Lambda_y = Lambda_z, Lambda_x = ratio Lambda_z at the filling
    factor of a sphere of radius Lambda/3 in a cube (f = 0.155)."""
    a = (4.0 * math.pi * radius ** 3 / (3.0 * f * ratio)) ** (1.0 / 3.0)
    return (ratio * a, a, a)


def orthorhombic_periods(ratio, radius, f=4.0 * math.pi / (81.0 * 1.1)):
    """Fig. 5: Lambda_y = 1.1 Lambda_z, Lambda_x = ratio Lambda_z at the
    filling factor of a sphere of radius Lambda_x/3 with Lambda_x = Lambda_z
    (f = 0.141)."""
    a = (4.0 * math.pi * radius ** 3 / (3.0 * f * ratio * 1.1)) ** (1.0 / 3.0)
    return (ratio * a, 1.1 * a, a)


def cavity_structure(periods, radius, n_host=N_HOST):
    """One air sphere at the cell centre of a matrix of index n_host."""
    c = tuple(p / 2.0 for p in periods)
    return dict(periods=tuple(periods), eps_host=n_host ** 2,
                shapes=[(wl.SPHERE, c, (radius, radius, radius), 1.0)])


def principal_indices(structure, n_harm, n_guess, k0=K0, rel=0.12, n_kappa=16, **plan_kw):
    """(n_x, n_y, n_z) = sqrt(eps_aa) of the principal sweeps, windows of
    +-rel around n_guess."""
    plan = gsm.plan_for(structure, n_harm, **plan_kw)
    try:
        win = [(k0 * n_guess * (1 - rel), k0 * n_guess * (1 + rel))] * 3
        eps, _ = plan.retrieve_tensor(k0, win, n_kappa=n_kappa)
    finally:
        plan.close()
    return np.sqrt(eps)


def mode_index(plan, kdir, pol, n_guess, k0=K0, rel=0.12, n_kappa=16, Np=5, Nd=10):
    """Mode index along an arbitrary direction: xi = a^H E_0 over an
    equidistant kappa grid (one gsm_sweep), the pole fit of Eqs. 7-10, and the
    largest-residue pole inside the grid."""
    kap = np.linspace(k0 * n_guess * (1 - rel), k0 * n_guess * (1 + rel), n_kappa)
    pts = [wl.point(kv, kdir, pol, k0) for kv in kap]
    E0, _ = plan.sweep(pts)
    a = np.asarray(pol, complex)
    xi = E0 @ np.conj(a)
    eta, zeta = gsm.fit_poles(kap, xi, Np, Nd)
    inside = [j for j in range(Np) if kap[0] <= eta[j].real <= kap[-1]]
    if not inside:
        raise RuntimeError("no pole inside the kappa window")
    j = max(inside, key=lambda j: abs(zeta[j]))
    return float(eta[j].real / k0)


def fresnel_xz(n, theta):
    """Normal-surface indices of an ideal biaxial medium with principal
    indices n = (n_x, n_y, n_z) for the direction s = (sin t, 0, cos t) in the
    xz plane: D along y gives n_y; D in the plane gives
    1 / n^2 = sin^2 t / n_z^2 + cos^2 t / n_x^2."""
    s, c = math.sin(theta), math.cos(theta)
    return n[1], 1.0 / math.sqrt(s * s / n[2] ** 2 + c * c / n[0] ** 2)


def normal_surface_xz(structure, n_harm, thetas, n_guess, k0=K0, **plan_kw):
    """Cross-section of the normal surface by the xz plane: for each angle
    the two mode indices (E along y, E in the plane perpendicular to s)."""
    plan = gsm.plan_for(structure, n_harm, **plan_kw)
    out = []
    try:
        for t in thetas:
            s = (math.sin(t), 0.0, math.cos(t))
            e_plane = (math.cos(t), 0.0, -math.sin(t))
            out.append((mode_index(plan, s, (0.0, 1.0, 0.0), n_guess, k0),
                        mode_index(plan, s, e_plane, n_guess, k0)))
    finally:
        plan.close()
    return np.array(out)


def figure(kind, n_harm=(9, 9, 9), ratios=(0.7, 0.85, 1.0, 1.15, 1.3), radii=RADII, **plan_kw):
    """Principal indices versus the period ratio for each cavity radius
    (Fig. 4a for kind "tetragonal", Fig. 5a for "orthorhombic")."""
    per = tetragonal_periods if kind == "tetragonal" else orthorhombic_periods
    f = 4.0 * math.pi / 81.0 if kind == "tetragonal" else 4.0 * math.pi / (81.0 * 1.1)
    n_mg = math.sqrt(maxwell_garnett(1.0, N_HOST ** 2, f))
    rows = []
    for r in radii:
        for t in ratios:
            P = per(t, r)
            n = principal_indices(cavity_structure(P, r), n_harm, n_mg, **plan_kw)
            rows.append(dict(radius=r, ratio=t, periods=P, n=[float(v) for v in n]))
    return dict(kind=kind, fill=f, n_mg=n_mg, n_harm=list(n_harm), rows=rows)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("which", choices=["fig4", "fig5"])
    ap.add_argument("--harm", type=int, default=9)
    ap.add_argument("--out", default=None)
    args = ap.parse_args()
    res = figure("tetragonal" if args.which == "fig4" else "orthorhombic", (args.harm,) * 3,
                 precision=gsm.FP32_REFINE, tol=1e-10, max_batch=64)
    text = json.dumps(res)
    if args.out:
        with open(args.out, "w") as fh:
            fh.write(text)
    print(text)


if __name__ == "__main__":
    main()
