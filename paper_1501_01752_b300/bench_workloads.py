"""Secondary measurements beside the headline bench (bench.py --workload ...):

matvec    the Eq. 4 product alone: woodpile 31^3 harmonics, 64^3 grid, 32
          instances per launch, complex64 and FP64; per-pass device time,
          algorithmic GB/s and matvecs/s (also the small, clean target for
          ncu captures of the three product kernels).
sweep     batched resonance sweep for the tensor retrieval: ellipsoid lattice
          (eps 6, semi-axes 0.4/0.3/0.2 Lambda), 16 frequencies
          Lambda/lambda = 0.10..0.40 x 16 kappa x 2 polarisations = 512 solves,
          truncation 15/21/31 harmonics per axis by frequency group, one
          gsm_sweep call, then the pole fits.
gyroid    one large near-resonance solve: gyroid g > 0.5 voxels (128^3,
          eps 12), Lambda = 0.4, 63^3 harmonics (750k unknowns), 128^3 grid,
          Krylov basis capped to 256 MB; complex64 + refinement and FP64.
adjoint   gradient of eps_xx - eps_yy with respect to 64^3 voxel
          permittivities (seeded mirror-symmetric random binary field,
          eps in {1, 6}, fill 0.3), 21^3 harmonics.
optimise  50 projected gradient steps on that objective.

Each prints one JSON line.  All inputs are synthetic (workloads.py).
"""
from __future__ import annotations

import json
import math
import time

import numpy as np
import torch

from . import gsm
from . import workloads as wl


def _mg(eps_i, eps_h, f):
    b = (eps_i - eps_h) / (eps_i + 2 * eps_h)
    return eps_h * (1 + 2 * f * b) / (1 - f * b)


def _window(k0, n, lo=0.85, hi=1.15):
    # stay clear of the basis light cone kappa = k0 (eps_b = 1)
    return max(n * lo, 1.03) * k0, n * hi * k0


def _pc(args):
    return gsm.PRECOND_NONE if getattr(args, "precond", "auto") == "none" else gsm.PRECOND_AUTO


def run(name, args):
    torch.cuda.init()
    {"matvec": matvec, "sweep": sweep, "gyroid": gyroid, "adjoint": adjoint, "optimise": optimise,
     "nearpole": nearpole}[name](args)


def _events():
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    return a, b


def matvec(args):
    peak = _hbm_peak()
    st = wl.woodpile()
    pts = wl.woodpile_batch(getattr(args, "mv_batch", 32))
    B, U = len(pts), 3 * 31 ** 3
    # a short restart keeps the Krylov workspace of the warm-up solve small
    plan = gsm.plan_for(st, (31, 31, 31), precision=gsm.FP32_REFINE, tol=1e-8, max_batch=B,
                        restart=60 if B <= 32 else 8)
    plan.solve(pts[:B])                       # builds the level and runs the block-size autotuner
    x = wl.random_field((31, 31, 31), 1501, B)
    xd = torch.from_numpy(x.reshape(B, U)).cuda()
    res = {"workload": "woodpile 31^3 harmonics, 64^3 grid, %d instances per product" % B,
           "autotuned_blocks": list(plan.tuned_blocks())}
    reps = max(3, int(getattr(args, "steps", 10)))
    for name, prec, pc in (("c64", gsm.FP32_REFINE, False), ("c64_precond", gsm.FP32_REFINE, True),
                           ("fp64", gsm.FP64, False)):
        for _ in range(3):
            plan.apply(pts, xd, precision=prec, precond=pc)
        plan.profile(True)
        for _ in range(reps):
            plan.apply(pts, xd, precision=prec, precond=pc)
        out = {}
        tot = 0.0
        for kname, kind in (("fwd_x", gsm.KIND_FWD_X), ("yz_conv", gsm.KIND_YZ), ("inv_x_green", gsm.KIND_INV_X)):
            n, ms, by = plan.profile_get(kind)
            tot += ms
            gbs = by / (ms * 1e-3) / 1e9 if ms > 0 else 0.0
            out[kname] = {"launches": n, "us_per_launch": 1e3 * ms / max(n, 1), "GB/s": gbs,
                          "frac_of_measured_hbm": gbs / peak}
        plan.profile(False)
        out["matvecs_per_s"] = B * reps / (tot * 1e-3)
        out["us_per_product_of_%d" % B] = 1e3 * tot / reps
        res[name] = out
    plan.close()
    print(json.dumps(res), flush=True)


def _hbm_peak():
    import os
    p = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            return float(json.load(f)["hbm_gbs"])
    except (OSError, KeyError, ValueError):
        return 6400.0


def sweep(args):
    print(json.dumps(sweep_c3(args)), flush=True)


def c3_points():
    """The C3 resonance sweep's points: the ellipsoid lattice (eps 6, Lambda
    = 1), 16 frequencies k0 Lambda / 2 pi = 0.10 ... 0.40 with truncations
    15/21/31 in turn, 16 kappa across each resonance window, x and y
    polarisation along z.  Returns (structure, points, groups, n_MG); each
    group is (ratio, polarisation, kappa values, point indices, k0)."""
    st = wl.ellipsoid_lattice(period=1.0)
    f = 4 * math.pi / 3 * 0.4 * 0.3 * 0.2
    n_mg = math.sqrt(_mg(6.0, 1.0, f))
    pts, groups = [], []
    for gi in range(16):
        ratio = 0.10 + 0.02 * gi
        k0 = 2 * math.pi * ratio                 # Lambda = 1
        N = (15, 21, 31)[gi % 3]
        lo, hi = _window(k0, n_mg)
        kap = np.linspace(lo, hi, 16)
        for pol in ((1, 0, 0), (0, 1, 0)):
            idx = []
            for kv in kap:
                p = wl.point(kv, (0, 0, 1), pol, k0)
                p["n_harm"] = (N, N, N)
                idx.append(len(pts))
                pts.append(p)
            groups.append((ratio, pol, kap, idx, k0))
    return st, pts, groups, n_mg


def sweep_c3(args):
    """The C3 resonance sweep of the retrieval, timed: gsm_sweep over the 512
    points of c3_points() (batches of sweep_batch points, which may span
    truncations), then the 32 pole fits on the host.  Returns the result as
    a dict."""
    st, pts, groups, n_mg = c3_points()
    mb = getattr(args, "sweep_batch", 256)
    plan = gsm.plan_for(st, (31, 31, 31), precision=gsm.FP32_REFINE, tol=1e-8, max_batch=mb, precond=_pc(args))
    plan.sweep(pts[:64])                          # warm-up (plan levels, workspaces)
    torch.cuda.synchronize()
    # the whole sweep five times (each call solves all 512 points from
    # scratch): the median, since one 0.1 s call is exposed to host jitter
    reps = []
    for _ in range(5):
        t0 = time.perf_counter()
        E0, infos = plan.sweep(pts)
        reps.append(time.perf_counter() - t0)
    t_sweep = float(np.median(reps))
    t0 = time.perf_counter()
    out = []
    for ratio, pol, kap, idx, k0 in groups:
        xi = np.array([np.vdot(np.asarray(pol, complex), E0[i]) for i in idx])
        eta, zeta = gsm.fit_poles(kap, xi, 5, 10)
        inside = [j for j in range(5) if kap[0] <= eta[j].real <= kap[-1]]
        j = max(inside, key=lambda j: abs(zeta[j])) if inside else None
        out.append(None if j is None else float(((eta[j] / k0) ** 2).real))
    t_fit = time.perf_counter() - t0
    iters = [i["iters"] for i in infos]
    plan.close()
    import os
    return {
        "workload": "sweep: ellipsoid lattice eps 6, 16 omega x 16 kappa x 2 pol, N = 15/21/31",
        "precond": getattr(args, "precond", "auto"), "max_batch": mb,
        "batches": "one truncation each" if os.environ.get("GSM_MIXED") == "0" else "across truncations",
        "solves": len(pts), "seconds": t_sweep, "seconds_each": reps, "solves_per_s": len(pts) / t_sweep,
        "retrieval_host_ms": 1000 * t_fit, "iters_mean": float(np.mean(iters)),
        "rel_residual_max": float(max(i["rel_residual"] for i in infos)),
        "eps_xx_by_ratio": out[0::2], "eps_yy_by_ratio": out[1::2], "n_MG": n_mg}


def gyroid(args):
    vox = wl.gyroid_voxels(128, 0.5, (1.0, 12.0))
    st = dict(periods=(0.4, 0.4, 0.4), voxels=vox)
    k0 = 2 * math.pi
    f = float(np.mean(vox > 2))
    n0 = math.sqrt(_mg(12.0, 1.0, f))
    # locate the x-polarised mode pole on a 15^3 truncation, then solve at 63^3
    # just above it (slow Krylov convergence near the resonance)
    coarse = gsm.plan_for(st, (15, 15, 15), precision=gsm.FP64, tol=1e-10)
    lo, hi = _window(k0, n0, 0.8, 1.3)
    eps, diag = coarse.retrieve_tensor(k0, [(lo, hi)] * 3, 16)
    eta = float(diag["eta"][0].real)
    coarse.close()
    pt = wl.point(eta * (1 + 1e-3), (0, 0, 1), (1, 0, 0), k0)
    res = {"workload": "gyroid g > 0.5 eps 12, Lambda 0.4, 63^3 harmonics, 128^3 grid, 256 MB Krylov cap",
           "fill": f, "kappa_over_k0": pt["kappa"] / k0, "eta15_over_k0": eta / k0,
           "precond": getattr(args, "precond", "auto")}
    U = 3 * 63 ** 3
    for name, prec in (("c64_refine", gsm.FP32_REFINE), ("fp64", gsm.FP64)):
        plan = gsm.plan_for(st, (63, 63, 63), precision=prec, tol=1e-8, max_batch=1, hbm_cap=256 << 20,
                            max_iter=20000, precond=_pc(args))
        E = torch.empty(U, dtype=torch.complex128, device="cuda")
        t = []
        for _ in range(2):   # the first solve also loads kernels, tunes block sizes and captures graphs
            a, b = _events()
            a.record()
            _, infos, s = plan.solve([pt], out=E)
            b.record()
            b.synchronize()
            t.append(a.elapsed_time(b) / 1000)
        res[name] = dict(seconds=t[1], first_solve_seconds=t[0], iters=infos[0]["iters"],
                         refine_steps=infos[0]["refine_steps"], rel_residual=infos[0]["rel_residual"],
                         status=infos[0]["status"])
        plan.close()
    print(json.dumps(res), flush=True)


NEARPOLE_DELTAS = (-1e-2, -1e-3, -1e-4, -1e-5, -1e-6, 1e-6, 1e-5, 1e-4, 1e-3, 1e-2)


def woodpile_pole(n_harm, k0=2 * math.pi):
    """The x-polarised mode pole eta of the woodpile along z at truncation
    n_harm: FP64 sweep over [1.5, 1.9] k0 and the Eqs. 7-10 fit."""
    plan = gsm.plan_for(wl.woodpile(), n_harm, precision=gsm.FP64, tol=1e-12)
    _, diag = plan.retrieve_tensor(k0, [(1.5 * k0, 1.9 * k0)] * 3, 16)
    plan.close()
    return float(diag["eta"][0].real)


def nearpole_solves(n_harm, eta, krylov, precision, tol, deltas=NEARPOLE_DELTAS, k0=2 * math.pi, max_iter=2000):
    """Solves of the woodpile at kappa = eta (1 + delta), x polarisation along z:
    the points around a mode pole where the paper finds that GMRES converges
    and other iterative methods fail ("Calculation details")."""
    pts = [wl.point(eta * (1 + d), (0, 0, 1), (1, 0, 0), k0) for d in deltas]
    plan = gsm.plan_for(wl.woodpile(), n_harm, precision=precision, tol=tol, max_batch=len(pts), max_iter=max_iter,
                        krylov=krylov)
    E, infos, s = plan.solve(pts)
    plan.close()
    return pts, E, infos


def nearpole(args):
    """GMRES against BiCGSTAB around the woodpile's x-polarised pole (15^3
    harmonics, 32^3 grid): products, refinement steps and status per point,
    complex64 + refinement (tol 1e-8) and FP64 (tol 1e-10)."""
    n_harm = (15, 15, 15)
    eta = woodpile_pole(n_harm)
    res = {"workload": "woodpile 15^3 harmonics, kappa = eta (1 + delta) around the x-polarised pole",
           "eta_over_k0": eta / (2 * math.pi), "deltas": list(NEARPOLE_DELTAS)}
    for kname, kr in (("gmres", gsm.GMRES), ("bicgstab", gsm.BICGSTAB)):
        for pname, prec, tol in (("c64_refine", gsm.FP32_REFINE, 1e-8), ("fp64", gsm.FP64, 1e-10)):
            t0 = time.perf_counter()
            _, _, infos = nearpole_solves(n_harm, eta, kr, prec, tol)
            res["%s_%s" % (kname, pname)] = {
                "seconds": time.perf_counter() - t0,
                "products": [i["iters"] for i in infos], "refine_steps": [i["refine_steps"] for i in infos],
                "status": [i["status"] for i in infos], "rel_residual": [i["rel_residual"] for i in infos]}
    print(json.dumps(res), flush=True)


def _c4():
    vox = wl.random_binary_voxels(64, 1501, 2.0, 0.3, (1.0, 6.0), mirror=True)
    st = dict(periods=(0.3, 0.3, 0.3), voxels=vox)
    k0 = 2 * math.pi
    n0 = math.sqrt(_mg(6.0, 1.0, 0.3))
    lo, hi = _window(k0, n0)
    return vox, st, k0, [(lo, hi)] * 3


def adjoint(args):
    vox, st, k0, win = _c4()
    plan = gsm.plan_for(st, (21, 21, 21), precision=gsm.FP32_REFINE, tol=1e-10, max_batch=64)
    plan.retrieve_tensor(k0, win, 16)
    a, b = _events()
    a.record()
    eps, grad = plan.retrieve_tensor_grad(k0, win, (1.0, -1.0, 0.0), 16)
    b.record()
    b.synchronize()
    print(json.dumps({"workload": "adjoint: 64^3 mirror-symmetric random voxels, 21^3 harmonics",
                      "seconds_per_gradient": a.elapsed_time(b) / 1000, "eps": list(map(float, eps)),
                      "grad_abs_max": float(np.abs(grad).max()), "grad_sum": float(grad.sum())}), flush=True)
    plan.close()


def optimise(args):
    from .autograd import optimise_anisotropy
    vox, st, k0, win = _c4()
    plan = gsm.plan_for(st, (21, 21, 21), precision=gsm.FP32_REFINE, tol=1e-10, max_batch=64)
    t0 = time.perf_counter()
    v, hist = optimise_anisotropy(plan, vox, k0, win, steps=max(1, args.steps))
    dt = time.perf_counter() - t0
    obj = hist[:, 0] - hist[:, 1]
    acc = hist[:, 3] > 0
    print(json.dumps({"workload": "optimise eps_xx - eps_yy, 64^3 voxels, 21^3 harmonics",
                      "evaluations": len(hist), "accepted": int(acc.sum()), "seconds": dt,
                      "objective_first": float(obj[0]), "objective_best": float(obj[acc].max()),
                      "objective": [round(float(o), 6) for o in obj], "accepted_flags": [int(a) for a in acc],
                      "eps_history": [[round(float(e), 6) for e in h[:3]] for h in hist]}),
          flush=True)
    plan.close()
