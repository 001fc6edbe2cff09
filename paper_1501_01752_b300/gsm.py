"""ctypes binding of the C ABI in ``include/gsm.h`` (argument marshalling only;
every step of the solve runs in ``libgsm.so``).

Host arrays are numpy; device arrays are torch CUDA tensors, passed by
pointer together with the plan's stream.  A missing library raises at import:
there is no fallback path.
"""
from __future__ import annotations

import ctypes as ct
import os

import numpy as np

from . import workloads as wl

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgsm.so")

GSM_OK, GSM_ERR_ARG, GSM_ERR_SINGULAR, GSM_ERR_NOCONV, GSM_ERR_NOMEM, GSM_ERR_CUDA, GSM_ERR_TIMEOUT, GSM_ERR_STATE = range(8)
STATUS_NAMES = ["GSM_OK", "GSM_ERR_ARG", "GSM_ERR_SINGULAR", "GSM_ERR_NOCONV", "GSM_ERR_NOMEM",
                "GSM_ERR_CUDA", "GSM_ERR_TIMEOUT", "GSM_ERR_STATE"]
FP64, FP32_REFINE = 0, 1
DF64 = 2                      # gsm_apply only: the double-float product (outer-residual arithmetic)
RESID_AUTO, RESID_FP64 = 0, 1
FORM_E, FORM_H = 0, 1         # Eq. 4 (E field) or Eq. 5 (H field)
GMRES, BICGSTAB = 0, 1
PRECOND_AUTO, PRECOND_NONE = 0, 1   # averaged-medium right preconditioner of GMRES on Eq. 4, or none
KIND_FWD_X, KIND_YZ, KIND_INV_X, KIND_DOTS, KIND_UPDATE, KIND_OTHER, KIND_RESID64, KIND_LAUNCHES = range(8)


class GsmError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES[status] if 0 <= status < 8 else status, msg))
        self.status = status


class PlanDesc(ct.Structure):
    _fields_ = [("period", ct.c_double * 3), ("n_harm", ct.c_int * 3), ("fft", ct.c_int * 3),
                ("eps_b", ct.c_double * 2), ("precision", ct.c_int), ("krylov", ct.c_int),
                ("restart", ct.c_int), ("max_iter", ct.c_int), ("tol", ct.c_double),
                ("inner_tol", ct.c_double), ("max_batch", ct.c_int), ("hbm_cap_bytes", ct.c_size_t),
                ("device", ct.c_int), ("cuda_stream", ct.c_void_p), ("residual", ct.c_int),
                ("form", ct.c_int), ("precond", ct.c_int)]


class Shape(ct.Structure):
    _fields_ = [("kind", ct.c_int), ("center", ct.c_double * 3), ("size", ct.c_double * 3),
                ("eps", ct.c_double * 2)]


class Point(ct.Structure):
    _fields_ = [("k0", ct.c_double), ("kdir", ct.c_double * 3), ("kappa", ct.c_double),
                ("pol", ct.c_double * 6), ("n_harm", ct.c_int * 3)]


class Info(ct.Structure):
    _fields_ = [("iters", ct.c_int), ("refine_steps", ct.c_int), ("rel_residual", ct.c_double),
                ("status", ct.c_int)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError("libgsm.so is not built (run python -m paper_1501_01752_b300.build)")
    lib = ct.CDLL(LIB_PATH)
    P = ct.c_void_p
    dp = ct.POINTER(ct.c_double)
    sig = {
        "gsm_plan_query": (ct.c_int, [ct.POINTER(PlanDesc), ct.POINTER(ct.c_int), ct.POINTER(ct.c_size_t)]),
        "gsm_plan": (ct.c_int, [ct.POINTER(PlanDesc), ct.POINTER(P)]),
        "gsm_plan_destroy": (None, [P]),
        "gsm_set_permittivity": (ct.c_int, [P, dp, ct.POINTER(Shape), ct.c_int, dp, ct.POINTER(ct.c_int)]),
        "gsm_apply": (ct.c_int, [P, ct.c_int, ct.POINTER(Point), P, P, ct.c_int, ct.c_int, ct.c_int]),
        "gsm_apply_noalloc": (ct.c_int, [P, ct.POINTER(Point), P, P]),
        "gsm_solve": (ct.c_int, [P, ct.c_int, ct.POINTER(Point), P, ct.c_int, ct.POINTER(Info)]),
        "gsm_sweep": (ct.c_int, [P, ct.c_int, ct.POINTER(Point), dp, ct.POINTER(Info)]),
        "gsm_fit_poles": (ct.c_int, [ct.c_int, dp, dp, ct.c_int, ct.c_int, dp, dp]),
        "gsm_retrieve_tensor": (ct.c_int, [P, ct.c_double, dp, ct.c_int, ct.c_int, ct.c_int, dp, dp]),
        "gsm_adjoint": (ct.c_int, [P, ct.c_int, ct.POINTER(Point), dp, dp]),
        "gsm_retrieve_tensor_grad": (ct.c_int, [P, ct.c_double, dp, ct.c_int, ct.c_int, ct.c_int, dp, dp, dp]),
        "gsm_profile": (ct.c_int, [P, ct.c_int]),
        "gsm_tuned_blocks": (ct.c_int, [P, ct.c_int, ct.POINTER(ct.c_int)]),
        "gsm_level_fft": (ct.c_int, [P, ct.POINTER(ct.c_int), ct.POINTER(ct.c_int)]),
        "gsm_profile_get": (ct.c_int, [P, ct.c_int, ct.POINTER(ct.c_longlong), dp, dp]),
        "gsm_probe_fma": (ct.c_int, [ct.c_int, P, ct.c_int, dp]),
        "gsm_last_error": (ct.c_char_p, [P]),
        "gsm_version": (ct.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


lib = _load()


def _dp(a):
    return a.ctypes.data_as(ct.POINTER(ct.c_double))


# numpy image of Point (C layout, 8-byte aligned): the points of a call are
# filled column by column, much faster than field-by-field ctypes stores
_POINT_DT = np.dtype([("k0", "<f8"), ("kdir", "<f8", 3), ("kappa", "<f8"), ("pol", "<f8", 6),
                      ("n_harm", "<i4", 3)], align=True)
assert _POINT_DT.itemsize == ct.sizeof(Point)


class _Points:
    """A contiguous gsm_point array that ctypes passes as Point* (numpy-backed)."""

    def __init__(self, arr):
        self.arr = arr
        self._as_parameter_ = arr.ctypes.data_as(ct.POINTER(Point))

    def __len__(self):
        return len(self.arr)


def make_points(points):
    """gsm_point array from dicts (k0, kdir, kappa, pol[, n_harm]) as made by
    workloads.point()."""
    n = len(points)
    arr = np.zeros(n, dtype=_POINT_DT)
    arr["k0"] = [p["k0"] for p in points]
    arr["kdir"] = [p["kdir"] for p in points]
    arr["kappa"] = [p["kappa"] for p in points]
    pol = np.array([p["pol"] for p in points], dtype=np.complex128).reshape(n, 3)
    arr["pol"] = pol.view(np.float64).reshape(n, 6)
    arr["n_harm"] = [p.get("n_harm", (0, 0, 0)) for p in points]
    return _Points(arr)


def fit_poles(kappa, xi, Np=5, Nd=10):
    """Eqs. 7-10 pole fit on the host (libgsm)."""
    kappa = np.ascontiguousarray(kappa, dtype=np.float64)
    xi = np.ascontiguousarray(np.asarray(xi, dtype=np.complex128)).view(np.float64)
    eta = np.zeros(2 * Np)
    zeta = np.zeros(2 * Np)
    s = lib.gsm_fit_poles(len(kappa), _dp(kappa), _dp(xi), Np, Nd, _dp(eta), _dp(zeta))
    if s:
        raise GsmError(s, "gsm_fit_poles")
    return eta.view(np.complex128), zeta.view(np.complex128)


def probe_fma(kind, device=0, stream=None):
    """Measured FMA throughput in TFLOP/s (gsm_probe_fma): kind 0 FP64,
    1 FP32, 2 packed FP32 pairs."""
    out = ct.c_double()
    s = lib.gsm_probe_fma(device, stream, kind, ct.byref(out))
    if s:
        raise GsmError(s, "gsm_probe_fma")
    return out.value


def plan_query(periods, n_harm, precision=FP32_REFINE, fft=(0, 0, 0), max_batch=0, restart=0, hbm_cap=0):
    d = _desc(periods, n_harm, 1.0, precision, restart, 0, 0, 0, max_batch, hbm_cap, 0, None, fft)
    L = (ct.c_int * 3)()
    nb = ct.c_size_t()
    s = lib.gsm_plan_query(ct.byref(d), L, ct.byref(nb))
    if s:
        raise GsmError(s, "gsm_plan_query")
    return tuple(L), nb.value


def _desc(periods, n_harm, eps_b, precision, restart, max_iter, tol, inner_tol, max_batch, hbm_cap, device,
          stream, fft, residual=RESID_AUTO, krylov=GMRES, form=FORM_E, precond=PRECOND_AUTO):
    d = PlanDesc()
    for a in range(3):
        d.period[a] = periods[a]
        d.n_harm[a] = n_harm[a]
        d.fft[a] = fft[a]
    d.eps_b[0] = float(np.real(eps_b))
    d.eps_b[1] = float(np.imag(eps_b))
    d.precision = precision
    d.krylov = krylov
    d.restart = restart
    d.max_iter = max_iter
    d.tol = tol
    d.inner_tol = inner_tol
    d.max_batch = max_batch
    d.hbm_cap_bytes = hbm_cap
    d.device = device
    d.cuda_stream = stream
    d.residual = residual
    d.form = form
    d.precond = precond
    return d


class Plan:
    """One structure truncation on one GPU (gsm_plan_t)."""

    def __init__(self, periods, n_harm, eps_b=1.0, precision=FP32_REFINE, restart=0, max_iter=0, tol=0.0,
                 inner_tol=0.0, max_batch=0, hbm_cap=0, device=0, stream=None, fft=(0, 0, 0), residual=RESID_AUTO,
                 krylov=GMRES, form=FORM_E, precond=PRECOND_AUTO):
        if stream is None:
            import torch
            stream = torch.cuda.current_stream(device).cuda_stream
        self.n_harm = tuple(n_harm)
        self.desc = _desc(periods, n_harm, eps_b, precision, restart, max_iter, tol, inner_tol, max_batch,
                          hbm_cap, device, stream, fft, residual, krylov, form, precond)
        h = ct.c_void_p()
        s = lib.gsm_plan(ct.byref(self.desc), ct.byref(h))
        if s:
            raise GsmError(s, "gsm_plan")
        self.h = h
        self.M = None

    def close(self):
        if getattr(self, "h", None):
            lib.gsm_plan_destroy(self.h)
            self.h = None

    def __del__(self):
        self.close()

    def _check(self, s, what):
        if s and s != GSM_ERR_NOCONV:
            raise GsmError(s, "%s: %s" % (what, lib.gsm_last_error(self.h).decode()))
        return s

    def set_permittivity(self, eps_host=1.0, shapes=(), voxels=None):
        eh = np.array([np.real(eps_host), np.imag(eps_host)], dtype=np.float64)
        arr = (Shape * max(1, len(shapes)))()
        for i, (kind, center, size, eps) in enumerate(shapes):
            arr[i].kind = kind
            for a in range(3):
                arr[i].center[a] = center[a]
                arr[i].size[a] = size[a]
            arr[i].eps[0] = np.real(eps)
            arr[i].eps[1] = np.imag(eps)
        if voxels is not None:
            v = np.ascontiguousarray(voxels, dtype=np.float64)   # [z][y][x]
            M = (ct.c_int * 3)(v.shape[2], v.shape[1], v.shape[0])
            self.M = v.shape
            s = lib.gsm_set_permittivity(self.h, _dp(eh), arr, 0, _dp(v), M)
        else:
            s = lib.gsm_set_permittivity(self.h, _dp(eh), arr, len(shapes), None, None)
        self._check(s, "gsm_set_permittivity")

    def set_structure(self, st):
        """Set eps(r) from a workloads.* structure dict."""
        self.set_permittivity(st.get("eps_host", 1.0), st.get("shapes", ()), st.get("voxels"))

    def field_size(self, point=None):
        N = self.n_harm
        if point is not None and point.get("n_harm"):
            N = point["n_harm"]
        return 3 * N[0] * N[1] * N[2]

    def apply(self, points, x, precision=FP64, adjoint=False, precond=False):
        """y = A x (A^H x with adjoint, A M^{-1} x with precond: the right-
        preconditioned operator of the Krylov solves) for n points; x of shape
        (n, 3, Nz, Ny, Nx) complex128, numpy (host) or torch CUDA tensor
        (device)."""
        op = 2 if precond else int(bool(adjoint))
        pts = make_points(points)
        dev = not isinstance(x, np.ndarray)
        if dev:
            import torch
            xin = x.contiguous()
            y = torch.empty_like(xin)
            s = lib.gsm_apply(self.h, len(points), pts, ct.c_void_p(xin.data_ptr()), ct.c_void_p(y.data_ptr()), 1,
                              precision, op)
        else:
            xin = np.ascontiguousarray(x, dtype=np.complex128)
            y = np.empty_like(xin)
            s = lib.gsm_apply(self.h, len(points), pts, ct.c_void_p(xin.ctypes.data), ct.c_void_p(y.ctypes.data), 0,
                              precision, op)
        self._check(s, "gsm_apply")
        return y

    def apply_noalloc(self, point, x, y):
        """y = A x for one point with the fixed-scratch FP64 product
        (gsm_apply_noalloc); x and y are torch CUDA complex128 tensors."""
        pts = make_points([point])
        s = lib.gsm_apply_noalloc(self.h, pts, ct.c_void_p(x.data_ptr()), ct.c_void_p(y.data_ptr()))
        self._check(s, "gsm_apply_noalloc")
        return y

    def solve(self, points, out=None, host_out=None):
        """Fields for n points: numpy (n, U) complex128 on the host, into a
        torch CUDA complex128 tensor `out`, or into a host (e.g. pinned) torch
        tensor `host_out`.  Returns (E, infos, status)."""
        pts = make_points(points)
        infos = (Info * len(points))()
        total = sum(self.field_size(p) for p in points)
        if out is not None:
            E = out
            s = lib.gsm_solve(self.h, len(points), pts, ct.c_void_p(out.data_ptr()), 1, infos)
        elif host_out is not None:
            E = host_out
            s = lib.gsm_solve(self.h, len(points), pts, ct.c_void_p(host_out.data_ptr()), 0, infos)
        else:
            E = np.zeros(total, dtype=np.complex128)
            s = lib.gsm_solve(self.h, len(points), pts, ct.c_void_p(E.ctypes.data), 0, infos)
        self._check(s, "gsm_solve")
        return E, [dict(iters=i.iters, refine_steps=i.refine_steps, rel_residual=i.rel_residual,
                        status=i.status) for i in infos], s

    def sweep(self, points):
        pts = make_points(points)
        infos = (Info * len(points))()
        E0 = np.zeros(6 * len(points))
        s = lib.gsm_sweep(self.h, len(points), pts, _dp(E0), infos)
        self._check(s, "gsm_sweep")
        return E0.view(np.complex128).reshape(len(points), 3), [
            dict(iters=i.iters, refine_steps=i.refine_steps, rel_residual=i.rel_residual, status=i.status)
            for i in infos]

    def retrieve_tensor(self, k0, windows, n_kappa=16, Np=5, Nd=10):
        lohi = np.ascontiguousarray(np.asarray(windows, dtype=np.float64).reshape(6))
        eps = np.zeros(3)
        diag = np.zeros(12)
        s = lib.gsm_retrieve_tensor(self.h, k0, _dp(lohi), n_kappa, Np, Nd, _dp(eps), _dp(diag))
        self._check(s, "gsm_retrieve_tensor")
        d = diag.reshape(3, 4)
        return eps, dict(eta=d[:, 0] + 1j * d[:, 1], zeta=d[:, 2] + 1j * d[:, 3])

    def adjoint(self, points, gE0):
        pts = make_points(points)
        g = np.ascontiguousarray(np.asarray(gE0, dtype=np.complex128).reshape(-1)).view(np.float64)
        out = np.zeros(int(np.prod(self.M)))
        s = lib.gsm_adjoint(self.h, len(points), pts, _dp(g), _dp(out))
        self._check(s, "gsm_adjoint")
        return out.reshape(self.M)

    def retrieve_tensor_grad(self, k0, windows, weights, n_kappa=16, Np=5, Nd=10):
        lohi = np.ascontiguousarray(np.asarray(windows, dtype=np.float64).reshape(6))
        w = np.ascontiguousarray(np.asarray(weights, dtype=np.float64))
        eps = np.zeros(3)
        out = np.zeros(int(np.prod(self.M)))
        s = lib.gsm_retrieve_tensor_grad(self.h, k0, _dp(lohi), n_kappa, Np, Nd, _dp(w), _dp(eps), _dp(out))
        self._check(s, "gsm_retrieve_tensor_grad")
        return eps, out.reshape(self.M)

    def level_fft(self, n_harm=None):
        """FFT grid of a built level (the tuned choice for fft = -1 axes)."""
        N = (ct.c_int * 3)(*(n_harm or self.n_harm))
        out = (ct.c_int * 3)()
        self._check(lib.gsm_level_fft(self.h, N, out), "gsm_level_fft")
        return tuple(out)

    def tuned_blocks(self, precision=FP32_REFINE):
        """Autotuned threads per block of the three product passes."""
        out = (ct.c_int * 3)()
        self._check(lib.gsm_tuned_blocks(self.h, precision, out), "gsm_tuned_blocks")
        return tuple(out)

    def profile(self, enable=True):
        self._check(lib.gsm_profile(self.h, int(enable)), "gsm_profile")

    def profile_get(self, kind):
        n = ct.c_longlong()
        ms = ct.c_double()
        by = ct.c_double()
        self._check(lib.gsm_profile_get(self.h, kind, ct.byref(n), ct.byref(ms), ct.byref(by)), "gsm_profile_get")
        return n.value, ms.value, by.value


def plan_for(structure, n_harm, **kw):
    """Plan + permittivity from a workloads.* structure dict."""
    p = Plan(structure["periods"], n_harm, **kw)
    p.set_structure(structure)
    return p


__all__ = ["Plan", "plan_for", "fit_poles", "plan_query", "make_points", "GsmError", "lib", "wl"]
