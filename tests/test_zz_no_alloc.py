"""gsm_apply_noalloc: the plan's operator (Eq. 4, or Eq. 5 for an H-field
plan) for callers that cannot allocate device memory during a solve step
(their own allocator has reserved the device up front, or an allocation's
implicit synchronisation is not acceptable).  It must give the same y = A x
as gsm_apply and as the oracle's FP64 operator, call after call, while every
temporary lives in the library's fixed device array.

Collected last on purpose (file name), so a stop-at-first-failure run has
run every other test before this one."""
import numpy as np
import pytest

from oracle import operator as oop
from paper_1501_01752_b300 import workloads as wl

from gpu_common import K0, gsm, oracle_structure, rel

pytestmark = pytest.mark.gpu


def test_noalloc_product_matches_gsm_apply_twice():
    import torch
    g = gsm()
    st = wl.woodpile()
    n_harm = (31, 31, 31)
    plan = g.plan_for(st, n_harm, precision=g.FP64)
    points = [wl.point(0.8 * K0), wl.point(0.73 * K0, (0.6, 0.0, 0.8), (0.0, 1.0, 0.0))]
    for i, pt in enumerate(points):                   # two calls in a row, different inputs
        x = wl.random_field(n_harm, 900 + i)
        want = plan.apply([pt], x[None])[0]          # the allocating entry point (host buffers)
        xd = torch.from_numpy(x).cuda()
        yd = torch.full_like(xd, complex(np.nan, np.nan))
        plan.apply_noalloc(pt, xd, yd)
        got = yd.cpu().numpy()
        assert np.all(np.isfinite(got))
        assert rel(got, want) < 1e-12, (i, rel(got, want))
    plan.close()


@pytest.mark.parametrize("form", ["E", "H"])
def test_noalloc_product_matches_oracle_operator_twice(form):
    # the oracle's FP64 operator of the same form (Eq. 4: E, Eq. 5: H) on a
    # small truncation, two calls in a row with different points and inputs
    import torch
    g = gsm()
    st = wl.random_shapes(3)
    n_harm = (7, 7, 7)
    ost = oracle_structure(st)
    H = form == "H"
    plan = g.plan_for(st, n_harm, precision=g.FP64, form=g.FORM_H if H else g.FORM_E)
    points = [wl.point(0.8 * K0, (0, 0, 1), (0, 1, 0)), wl.point(0.71 * K0, (0.3, -0.2, 0.9), (0.2, 0.5, 0.1j))]
    for i, pt in enumerate(points):
        x = wl.random_field(n_harm, 950 + i)
        kinc = pt["kappa"] * np.asarray(pt["kdir"])
        if H:
            A = oop.OperatorH(ost.delta_h(n_harm, 1.0), n_harm, kinc, st["periods"], pt["k0"] ** 2)
        else:
            A = oop.Operator(ost.delta(n_harm, 1.0), n_harm, kinc, st["periods"], pt["k0"] ** 2)
        want = A(x.reshape((3,) + n_harm[::-1])).ravel()
        xd = torch.from_numpy(x).cuda()
        yd = torch.full_like(xd, complex(np.nan, np.nan))
        plan.apply_noalloc(pt, xd, yd)
        got = yd.cpu().numpy().ravel()
        assert np.all(np.isfinite(got))
        assert rel(got, want) < 1e-12, (form, i, rel(got, want))
    plan.close()


def test_noalloc_rejects_oversized_truncation():
    import torch
    g = gsm()
    st = wl.woodpile()
    n_harm = (63, 63, 63)       # 3 * 128 * 63 * 63 complex128 temporaries: more than the fixed array
    plan = g.plan_for(st, n_harm, precision=g.FP64)
    x = torch.zeros((3,) + n_harm[::-1], dtype=torch.complex128, device="cuda")
    y = torch.empty_like(x)
    with pytest.raises(g.GsmError) as ei:
        plan.apply_noalloc(wl.point(0.8 * K0), x, y)
    assert ei.value.status == g.GSM_ERR_ARG and "scratch" in str(ei.value)
    plan.close()
