"""torch.autograd wrapper of the retrieved effective tensor: eps_eff(voxel eps).

Forward: gsm_retrieve_tensor (three principal resonance sweeps, pole fit).
Backward: gsm_retrieve_tensor_grad with the incoming gradient as weights
(adjoint solves on the GPU, pole sensitivities on the host).  The voxel
tensor lives on the CPU (it is copied into the plan's Fourier coefficients);
every solve runs in libgsm on the plan's device.
"""
from __future__ import annotations

import numpy as np
import torch

from . import gsm


class EffectiveTensor(torch.autograd.Function):
    """eps = EffectiveTensor.apply(voxels, plan, k0, windows, n_kappa, Np, Nd)

    voxels: float64 tensor [M_z, M_y, M_x] of real permittivities.
    Returns a float64 tensor (eps_xx, eps_yy, eps_zz)."""

    @staticmethod
    def forward(ctx, voxels, plan, k0, windows, n_kappa=16, Np=5, Nd=10):
        v = voxels.detach().cpu().double().numpy()
        plan.set_permittivity(voxels=v)
        eps, _ = plan.retrieve_tensor(k0, windows, n_kappa, Np, Nd)
        ctx.save_for_backward(voxels)
        ctx.args = (plan, k0, windows, n_kappa, Np, Nd)
        return torch.as_tensor(eps, dtype=torch.float64)

    @staticmethod
    def backward(ctx, grad_out):
        (voxels,) = ctx.saved_tensors
        plan, k0, windows, n_kappa, Np, Nd = ctx.args
        plan.set_permittivity(voxels=voxels.detach().cpu().double().numpy())
        w = grad_out.detach().cpu().double().numpy()
        _, g = plan.retrieve_tensor_grad(k0, windows, w, n_kappa, Np, Nd)
        return torch.as_tensor(g, dtype=voxels.dtype, device=voxels.device), None, None, None, None, None, None


def effective_tensor(voxels, plan, k0, windows, n_kappa=16, Np=5, Nd=10):
    return EffectiveTensor.apply(voxels, plan, k0, windows, n_kappa, Np, Nd)


def follow_windows(eps, k0, rel=0.15, floor=1.03):
    """kappa windows k0 sqrt(eps_cc) [1 - rel, 1 + rel] around the indices of
    the previous step (each lower end kept at floor k0, clear of the basis
    light cone kappa = k0 sqrt(eps_b) with eps_b = 1), so that every step
    retrieves the pole of the same mode while the structure changes."""
    n = np.sqrt(np.maximum(np.asarray(eps, dtype=np.float64), 1.0))
    return np.stack([np.maximum(n * (1 - rel), floor) * k0, n * (1 + rel) * k0], axis=1)


def optimise_anisotropy(plan, voxels, k0, windows, steps=50, lr=0.05, eps_range=(1.0, 6.0), log=None):
    """Projected gradient ascent of eps_xx - eps_yy over voxel permittivities
    kept in eps_range (the composite-design use of the adjoint), with step
    halving: a step that lowers the objective is undone and retried at half
    the length.  The first evaluation uses `windows`; later ones centre each
    component's window on the index of the last accepted structure
    (follow_windows).  `steps` counts evaluations (one retrieval each, plus
    one gradient per accepted step).  Returns the final voxels and the
    history of (eps_xx, eps_yy, eps_zz, accepted) per evaluation."""
    best_v = torch.tensor(np.asarray(voxels, dtype=np.float64))
    best_obj, best_g = None, None
    v = best_v.clone().requires_grad_(True)
    hist = []
    win = np.asarray(windows, dtype=np.float64)
    for it in range(steps):
        eps = effective_tensor(v, plan, k0, win)
        obj = float(eps[0] - eps[1])
        ok = best_obj is None or obj >= best_obj
        if ok:
            (g,) = torch.autograd.grad(eps[0] - eps[1], v)
            best_v, best_obj, best_g = v.detach().clone(), obj, g
            win = follow_windows(eps.detach().numpy(), k0)
        else:
            lr *= 0.5
        hist.append(np.append(eps.detach().numpy(), float(ok)))
        with torch.no_grad():
            scale = lr * (eps_range[1] - eps_range[0]) / max(float(best_g.abs().max()), 1e-30)
            v = (best_v + scale * best_g).clamp_(*eps_range).requires_grad_(True)
        if log:
            log(it, hist[-1])
    return best_v.numpy(), np.array(hist)
