"""The composite-design gradient through torch.autograd (EffectiveTensor):
d(eps_xx - eps_yy)/d(voxel eps) of the retrieved effective tensor.  The paper
has no adjoint; the checks are the oracle's explicit adjoint on a small cell,
the C entry point it wraps, central finite differences of the CUDA retrieval
at 32 seeded voxels of the 64^3-voxel, 21^3-harmonic configuration, and a
50-step projected gradient ascent on that configuration."""
import numpy as np
import pytest

from oracle import adjoint as oadj
from oracle import retrieval as ort
from paper_1501_01752_b300 import workloads as wl

from gpu_common import K0, gsm, rel

pytestmark = pytest.mark.gpu


def _small_cell():
    vox = wl.random_binary_voxels(M=8, seed=3, sigma=1.0, fill=0.3, mirror=True)
    periods = (0.25, 0.25, 0.25)
    f = float(np.mean(vox > 2))
    n0 = np.sqrt(ort.maxwell_garnett(6.0, 1.0, f))
    win = np.array([(K0 * n0 * 0.85, K0 * n0 * 1.15)] * 3)
    return vox, periods, win


def _c4():
    # the 64^3 seeded voxel field (seed 1501, sigma 2, fill 0.3, eps in {1, 6},
    # mirror-symmetric), Lambda = 0.3, windows around the Maxwell-Garnett index
    from paper_1501_01752_b300.bench_workloads import _c4 as c4
    vox, st, k0, win = c4()
    return vox, st, k0, np.array(win)


def test_effective_tensor_backward_is_retrieve_tensor_grad():
    import torch
    from paper_1501_01752_b300.autograd import effective_tensor
    g = gsm()
    vox, periods, win = _small_cell()
    plan = g.plan_for(dict(periods=periods, voxels=vox), (5, 5, 5), precision=g.FP64, tol=1e-13)
    v = torch.tensor(vox, requires_grad=True)
    eps = effective_tensor(v, plan, K0, win)
    w = torch.tensor([0.7, -1.3, 0.4], dtype=torch.float64)
    (gv,) = torch.autograd.grad((eps * w).sum(), v)
    eps_c, grad_c = plan.retrieve_tensor_grad(K0, win, w.numpy())
    assert np.array_equal(eps.detach().numpy(), eps_c)
    assert np.array_equal(gv.numpy(), grad_c)
    plan.close()


@pytest.mark.parametrize("prec", ["fp64", "c64_refine"])
def test_effective_tensor_gradient_matches_oracle(prec):
    import torch
    from paper_1501_01752_b300.autograd import effective_tensor
    g = gsm()
    vox, periods, win = _small_cell()
    n_harm = (5, 5, 5)
    fp64 = prec == "fp64"
    plan = g.plan_for(dict(periods=periods, voxels=vox), n_harm, precision=g.FP64 if fp64 else g.FP32_REFINE,
                      tol=1e-13 if fp64 else 1e-11)
    v = torch.tensor(vox, requires_grad=True)
    eps = effective_tensor(v, plan, K0, win)
    (gv,) = torch.autograd.grad(eps[0] - eps[1], v)
    ost = ort.Structure(periods, voxels=vox)
    kap = np.linspace(win[0][0], win[0][1], 16)
    exx, gxx = oadj.component_gradient(ost, n_harm, 1.0, K0, (0, 0, 1), (1, 0, 0), kap)
    eyy, gyy = oadj.component_gradient(ost, n_harm, 1.0, K0, (0, 0, 1), (0, 1, 0), kap)
    assert abs(float(eps[0]) - exx.real) < 1e-6 and abs(float(eps[1]) - eyy.real) < 1e-6
    assert rel(gv.numpy(), gxx - gyy) < 1e-5, rel(gv.numpy(), gxx - gyy)
    plan.close()


def test_c4_gradient_central_differences_at_32_voxels():
    # FP64 solves to 1e-13 keep the retrieval smooth to ~1e-13 relative, far
    # below the 2 h |dF/d eps_v| ~ 1e-9 that a central difference with
    # h = 1e-4 resolves on a 64^3 grid (per-voxel gradients ~1e-5)
    import torch
    from paper_1501_01752_b300.autograd import effective_tensor
    g = gsm()
    vox, st, k0, win = _c4()
    plan = g.plan_for(st, (21, 21, 21), precision=g.FP64, tol=1e-13, max_batch=64)
    v = torch.tensor(vox, requires_grad=True)
    eps = effective_tensor(v, plan, k0, win)
    (gv,) = torch.autograd.grad(eps[0] - eps[1], v)
    grad = gv.numpy()
    assert np.all(np.isfinite(grad))
    # the complex64 + refinement gradient of the same configuration
    pr = g.plan_for(st, (21, 21, 21), precision=g.FP32_REFINE, tol=1e-10, max_batch=64)
    _, g32 = pr.retrieve_tensor_grad(k0, win, (1.0, -1.0, 0.0))
    pr.close()
    assert rel(g32, grad) < 1e-4, rel(g32, grad)
    rng = np.random.Generator(np.random.PCG64(1501))
    flat = rng.choice(vox.size, size=32, replace=False)
    h = 1e-4
    gmax = float(np.max(np.abs(grad)))
    fds, ads = [], []
    for f in flat:
        idx = np.unravel_index(f, vox.shape)
        vals = []
        for sgn in (1.0, -1.0):
            vv = vox.copy()
            vv[idx] += sgn * h
            plan.set_permittivity(voxels=vv)
            e, _ = plan.retrieve_tensor(k0, win, 16)
            vals.append(e[0] - e[1])
        fds.append((vals[0] - vals[1]) / (2 * h))
        ads.append(grad[idx])
    fds, ads = np.array(fds), np.array(ads)
    err = np.abs(fds - ads)
    assert np.all(err < 1e-3 * gmax), (err.max() / gmax, fds, ads)
    assert rel(fds, ads) < 1e-3, rel(fds, ads)
    plan.close()


def test_c4_fifty_optimisation_steps_raise_the_anisotropy():
    from paper_1501_01752_b300.autograd import optimise_anisotropy
    g = gsm()
    vox, st, k0, win = _c4()
    plan = g.plan_for(st, (21, 21, 21), precision=g.FP32_REFINE, tol=1e-10, max_batch=64)
    v, hist = optimise_anisotropy(plan, vox, k0, win, steps=50)
    assert hist.shape == (50, 4) and np.all(np.isfinite(hist))
    assert np.all((v >= 1.0) & (v <= 6.0))
    obj = hist[:, 0] - hist[:, 1]
    acc = hist[:, 3] > 0
    best = np.maximum.accumulate(np.where(acc, obj, -np.inf))
    # ascent: accepted objectives never decrease, most steps are accepted,
    # and the anisotropy ends well above the starting one
    assert np.all(np.diff(obj[acc]) >= 0), obj
    assert acc.sum() >= 30, acc
    assert best[-1] > obj[0] + 0.1, obj
    # every accepted step retrieves the same modes: no index jumps by more than 10%
    na = np.sqrt(hist[acc, :3])
    assert np.all(np.abs(np.diff(na, axis=0)) < 0.1 * na[1:]), na
    plan.close()
