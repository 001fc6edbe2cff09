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


def optimise_anisotropy(plan, voxels, k0, windows, steps=50, lr=0.05, eps_range=(1.0, 6.0), log=None):
    """Projected gradient ascent of eps_xx - eps_yy over voxel permittivities
    kept in eps_range (the composite-design use of the adjoint).  Returns the
    final voxels and the history of (eps_xx, eps_yy, eps_zz)."""
    v = torch.tensor(np.asarray(voxels, dtype=np.float64), requires_grad=True)
    hist = []
    for it in range(steps):
        eps = effective_tensor(v, plan, k0, windows)
        obj = eps[0] - eps[1]
        (g,) = torch.autograd.grad(obj, v)
        with torch.no_grad():
            scale = lr * (eps_range[1] - eps_range[0]) / max(float(g.abs().max()), 1e-30)
            v += scale * g
            v.clamp_(*eps_range)
        hist.append(eps.detach().numpy().copy())
        if log:
            log(it, hist[-1])
    return v.detach().numpy(), np.array(hist)
