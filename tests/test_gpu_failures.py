"""Failure statuses of the C ABI, provoked on the host side (bad inputs,
impossible memory caps, calls out of order, iteration limits): no fault, trap
or hang is ever caused on the GPU."""
import numpy as np
import pytest

from paper_1501_01752_b300 import workloads as wl

from gpu_common import K0, gsm

pytestmark = pytest.mark.gpu


def test_solve_before_permittivity_is_a_state_error():
    g = gsm()
    plan = g.Plan((0.3, 0.3, 0.3), (5, 5, 5), precision=g.FP64)
    with pytest.raises(g.GsmError) as ei:
        plan.solve([wl.point(0.8 * K0)])
    assert ei.value.status == g.GSM_ERR_STATE
    plan.close()


def test_bad_inputs_are_argument_errors():
    g = gsm()
    plan = g.Plan((0.3, 0.3, 0.3), (5, 5, 5), precision=g.FP64)
    with pytest.raises(g.GsmError) as ei:
        plan.set_permittivity(2.0 + 0.1j)                  # lossy host: not supported
    assert ei.value.status == g.GSM_ERR_ARG
    vox = np.ones((4, 4, 4))
    vox[1, 2, 3] = np.nan                                  # non-finite voxel value
    with pytest.raises(g.GsmError) as ei:
        plan.set_permittivity(voxels=vox)
    assert ei.value.status == g.GSM_ERR_ARG
    plan.set_structure(wl.sphere_lattice())
    p = wl.point(0.8 * K0)
    p["n_harm"] = (7, 5, 5)                                # larger than the plan's truncation
    with pytest.raises(g.GsmError) as ei:
        plan.solve([p])
    assert ei.value.status == g.GSM_ERR_ARG
    p = dict(wl.point(0.8 * K0), kdir=(0.0, 0.0, 0.0))     # no direction
    with pytest.raises(g.GsmError) as ei:
        plan.solve([p])
    assert ei.value.status == g.GSM_ERR_ARG
    plan.close()


def test_memory_cap_too_small_is_nomem():
    g = gsm()
    U = 3 * 7**3
    plan = g.plan_for(wl.sphere_lattice(), (7, 7, 7), precision=g.FP32_REFINE, hbm_cap=2 * U * 8, max_batch=1)
    with pytest.raises(g.GsmError) as ei:
        plan.solve([wl.point(0.8 * K0)])
    assert ei.value.status == g.GSM_ERR_NOMEM
    plan.close()


def test_iteration_limit_returns_best_iterate_for_every_instance():
    g = gsm()
    plan = g.plan_for(wl.woodpile(), (15, 15, 15), precision=g.FP32_REFINE, tol=1e-12, max_iter=6, restart=6)
    pts = [wl.point(0.8 * K0), wl.point(0.75 * K0, pol=(0, 1, 0))]
    E, infos, s = plan.solve(pts)
    assert s == g.GSM_ERR_NOCONV
    for inf in infos:
        assert inf["status"] == g.GSM_ERR_NOCONV and inf["iters"] >= 6 and inf["rel_residual"] < 1.0
    assert np.all(np.isfinite(E))
    plan.close()
