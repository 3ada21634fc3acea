"""Python binding of libcsgb (circulant LASSO recovery on GB300).

Argument marshalling only: every step of ISTA / ADMM runs in the CUDA
library.  The names are those of the C ABI in ``include/cs.h``.  Device
vectors may be given as torch CUDA tensors (float32, contiguous) or as raw
device addresses (int); host arrays (rows, c) as numpy arrays.

The library is required: importing this package on a machine where
``libcsgb.so`` has not been built raises ``ImportError`` (there is no CPU
fallback).
"""
from __future__ import annotations

import ctypes
import math
import pathlib

import numpy as np

_PKG = pathlib.Path(__file__).resolve().parent
LIB_PATH = _PKG / "libcsgb.so"

CS_OK, CS_ERR_ARG, CS_ERR_NOMEM, CS_ERR_CUDA, CS_ERR_TIMEOUT, CS_ERR_NONFINITE, CS_ERR_UNSUPPORTED = range(7)

EXPORTS = ("cs_plan", "cs_plan_destroy", "cs_opnorm2", "cs_forward", "cs_adjoint",
           "cs_set_monitor", "cs_ista", "cs_admm", "cs_admm_ex", "cs_status_sync",
           "cs_status_string", "cs_version", "cs_profile_pass", "cs_circulant_apply_static",
           "cs_batch_plan", "cs_batch_destroy", "cs_batch_ista", "cs_batch_admm", "cs_batch_status_sync",
           "cs_grad", "cs_forward_direct", "cs_plan_2d", "cs_grad_admm")


class CsStats(ctypes.Structure):
    _fields_ = [("iters_run", ctypes.c_int), ("converged", ctypes.c_int),
                ("nmse", ctypes.c_double), ("rel_change", ctypes.c_double),
                ("objective", ctypes.c_double), ("ms", ctypes.c_double),
                ("launches", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class CsAdmmParams(ctypes.Structure):
    _fields_ = [("sigma", ctypes.c_double), ("rho", ctypes.c_double),
                ("tau1", ctypes.c_double), ("tau2", ctypes.c_double)]


class CsError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {status_string(code)} ({code})")


def _load() -> ctypes.CDLL:
    if not LIB_PATH.exists():
        raise ImportError(f"{LIB_PATH} is missing: build it with __graft_entry__.build() "
                          "(the CUDA library is required; there is no CPU fallback)")
    lib = ctypes.CDLL(str(LIB_PATH))
    vp, i64, f32, f64, ci = ctypes.c_void_p, ctypes.c_int64, ctypes.c_float, ctypes.c_double, ctypes.c_int
    sig = {
        "cs_plan": [ctypes.POINTER(vp), i64, i64, vp, vp, vp],
        "cs_plan_destroy": [vp],
        "cs_opnorm2": [vp, ci, ctypes.POINTER(f64)],
        "cs_forward": [vp, vp, vp],
        "cs_adjoint": [vp, vp, vp],
        "cs_set_monitor": [vp, vp, f64, ci],
        "cs_ista": [vp, vp, f32, f32, ci, vp, ctypes.POINTER(CsStats)],
        "cs_admm": [vp, vp, f32, f32, ci, vp, ctypes.POINTER(CsStats)],
        "cs_admm_ex": [vp, vp, f32, ctypes.POINTER(CsAdmmParams), ci, ci, vp, vp, vp, vp, vp,
                       ctypes.POINTER(CsStats)],
        "cs_status_sync": [vp],
        "cs_profile_pass": [vp, ci, ci],
        "cs_circulant_apply_static": [i64, vp, vp, vp, ci, vp],
        "cs_grad": [vp, vp, f32, f32, ci, ci, vp, vp, vp, vp],
        "cs_grad_admm": [vp, vp, f32, ctypes.POINTER(CsAdmmParams), ci, ci, vp, vp, vp, vp, vp],
        "cs_plan_2d": [ctypes.POINTER(vp), i64, i64, i64, vp, vp, vp],
        "cs_forward_direct": [i64, i64, vp, vp, vp, vp, vp],
        "cs_batch_plan": [ctypes.POINTER(vp), ci, vp, vp, vp, vp, vp],
        "cs_batch_destroy": [vp],
        "cs_batch_ista": [vp, vp, vp, vp, ci, vp],
        "cs_batch_admm": [vp, vp, vp, vp, ci, vp],
        "cs_batch_status_sync": [vp],
        "cs_status_string": [ci],
        "cs_version": [],
    }
    for name, args in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = ctypes.c_int
    lib.cs_status_string.restype = ctypes.c_char_p
    return lib


_lib = _load()


def status_string(code: int) -> str:
    return _lib.cs_status_string(int(code)).decode()


def cs_version() -> int:
    return int(_lib.cs_version())


def _ptr(t, dtype: str = "torch.float32", numel: int | None = None) -> int | None:
    """Device address of a tensor-like (torch tensor, int, None).  A tensor
    must be a contiguous CUDA tensor of `dtype` holding at least `numel`
    elements (when given); a raw int address is passed through unchecked."""
    if t is None:
        return None
    if isinstance(t, int):
        return t
    if hasattr(t, "data_ptr"):
        if getattr(t, "dtype", None) is not None and str(t.dtype) != dtype:
            raise TypeError(f"expected {dtype.split('.')[-1]}, got {t.dtype}")
        if hasattr(t, "is_contiguous") and not t.is_contiguous():
            raise ValueError("expected a contiguous tensor")
        if hasattr(t, "is_cuda") and not t.is_cuda:
            raise ValueError("expected a CUDA tensor")
        if numel is not None and t.numel() < numel:
            raise ValueError(f"expected at least {numel} elements, got {t.numel()}")
        return int(t.data_ptr())
    raise TypeError(f"cannot take a device pointer of {type(t)!r}")


def _check(code: int, where: str):
    if code != CS_OK:
        raise CsError(code, where)


def _stream_handle(stream) -> int | None:
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)


class Plan:
    """Owns a cs_plan_t; closes it on ``close()`` or garbage collection."""

    def __init__(self, handle: int, n: int, m: int):
        self.handle = handle
        self.n = n
        self.m = m

    def close(self):
        if self.handle:
            _lib.cs_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def cs_plan(n: int, m: int, rows, c, stream=None) -> Plan:
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    c = np.ascontiguousarray(c, dtype=np.float64)
    if rows.shape != (m,) or c.shape != (n,):
        raise ValueError("rows must have shape (m,) and c shape (n,)")
    h = ctypes.c_void_p()
    code = _lib.cs_plan(ctypes.byref(h), n, m, rows.ctypes.data, c.ctypes.data, _stream_handle(stream))
    _check(code, "cs_plan")
    return Plan(h.value, n, m)


def cs_plan_2d(n0: int, n1: int, m: int, pix, c2, stream=None) -> Plan:
    """Plan of the 2D blur A = P H of an n0 x n1 image (flattened row-major);
    pix: int64 (m,) kept pixels, c2: float64 (n0, n1) generating array."""
    pix = np.ascontiguousarray(pix, dtype=np.int64)
    c2 = np.ascontiguousarray(c2, dtype=np.float64)
    if pix.shape != (m,) or c2.shape != (n0, n1):
        raise ValueError("pix must have shape (m,) and c2 shape (n0, n1)")
    h = ctypes.c_void_p()
    code = _lib.cs_plan_2d(ctypes.byref(h), n0, n1, m, pix.ctypes.data, c2.ctypes.data, _stream_handle(stream))
    _check(code, "cs_plan_2d")
    return Plan(h.value, n0 * n1, m)


def cs_plan_destroy(plan: Plan):
    plan.close()


def cs_opnorm2(plan: Plan, iters: int = 100) -> float:
    L = ctypes.c_double()
    _check(_lib.cs_opnorm2(plan.handle, iters, ctypes.byref(L)), "cs_opnorm2")
    return L.value


def cs_forward(plan: Plan, x, y):
    _check(_lib.cs_forward(plan.handle, _ptr(x, numel=plan.n), _ptr(y, numel=plan.m)), "cs_forward")


def cs_adjoint(plan: Plan, r, x):
    _check(_lib.cs_adjoint(plan.handle, _ptr(r, numel=plan.m), _ptr(x, numel=plan.n)), "cs_adjoint")


def cs_set_monitor(plan: Plan, x_true=None, nmse_tol: float = 0.0, check_every: int = 10):
    _check(_lib.cs_set_monitor(plan.handle, _ptr(x_true, numel=plan.n), float(nmse_tol), int(check_every)),
           "cs_set_monitor")


def cs_ista(plan: Plan, y, lam: float, tau: float, iters: int, x, stats: bool = True):
    st = CsStats()
    code = _lib.cs_ista(plan.handle, _ptr(y, numel=plan.m), lam, tau, iters, _ptr(x, numel=plan.n),
                        ctypes.byref(st) if stats else None)
    _check(code, "cs_ista")
    return st.as_dict() if stats else None


def cs_admm(plan: Plan, y, lam: float, rho: float, iters: int, z, stats: bool = True):
    st = CsStats()
    code = _lib.cs_admm(plan.handle, _ptr(y, numel=plan.m), lam, rho, iters, _ptr(z, numel=plan.n),
                        ctypes.byref(st) if stats else None)
    _check(code, "cs_admm")
    return st.as_dict() if stats else None


def cs_admm_ex(plan: Plan, y, lam: float, sigma: float, rho: float, tau1: float, tau2: float,
               iters: int, warm: bool, x, z, mu, nu, v, stats: bool = True):
    st = CsStats()
    prm = CsAdmmParams(sigma, rho, tau1, tau2)
    n = plan.n
    code = _lib.cs_admm_ex(plan.handle, _ptr(y, numel=plan.m), lam, ctypes.byref(prm), iters, int(bool(warm)),
                           _ptr(x, numel=n), _ptr(z, numel=n), _ptr(mu, numel=n), _ptr(nu, numel=n),
                           _ptr(v, numel=n),
                           ctypes.byref(st) if stats else None)
    _check(code, "cs_admm_ex")
    return st.as_dict() if stats else None


def cs_grad(plan: Plan, y, lam: float, tau: float, T: int, K: int, gx_T, dc, dlam, dy):
    """Reverse mode of T ISTA steps from x(0) = 0: dc, dlam (1 element) and
    dy receive dL/dc, dL/dlambda, dL/dy for gx_T = dL/dx(T)."""
    n, m = plan.n, plan.m
    _check(_lib.cs_grad(plan.handle, _ptr(y, numel=m), lam, tau, int(T), int(K), _ptr(gx_T, numel=n),
                        _ptr(dc, numel=n), _ptr(dlam, numel=1), _ptr(dy, numel=m)), "cs_grad")


def cs_grad_admm(plan: Plan, y, lam: float, sigma: float, rho: float, tau1: float, tau2: float, T: int, K: int,
                 gz_T, dc, dlam, dy, gx_T=None):
    """Reverse mode of T iterations of Algorithm 3 from the zero state: dc,
    dlam (1 element) and dy receive dL/dc, dL/dlambda, dL/dy for gz_T =
    dL/dz(T) (and gx_T = dL/dx(T) when the loss also depends on x(T))."""
    prm = CsAdmmParams(sigma, rho, tau1, tau2)
    n, m = plan.n, plan.m
    _check(_lib.cs_grad_admm(plan.handle, _ptr(y, numel=m), lam, ctypes.byref(prm), int(T), int(K),
                             _ptr(gz_T, numel=n), _ptr(gx_T, numel=n), _ptr(dc, numel=n), _ptr(dlam, numel=1),
                             _ptr(dy, numel=m)), "cs_grad_admm")


def _make_unrolled_ista():
    import torch

    class UnrolledISTA(torch.autograd.Function):
        """x(T) of T ISTA steps from x(0) = 0, differentiable in c, y and lam.

        apply(c, y, lam, rows, tau, T, K): c float64 (n,) tensor (any device;
        a plan is made from it), y float32 CUDA (m,), lam a 0-d tensor or
        float, rows int64 (m,) array; tau, T, K plain numbers.  Forward runs
        cs_ista, backward cs_grad (checkpoints every K steps)."""

        @staticmethod
        def forward(ctx, c, y, lam, rows, tau, T, K):
            lam_f = float(lam)
            n, m = int(c.shape[0]), int(y.shape[0])
            stream = torch.cuda.current_stream(y.device)
            plan = cs_plan(n, m, np.asarray(rows), c.detach().double().cpu().numpy(), stream)
            x = torch.zeros(n, dtype=torch.float32, device=y.device)
            cs_ista(plan, y.detach().contiguous(), lam_f, float(tau), int(T), x, stats=False)
            ctx.plan, ctx.args = plan, (lam_f, float(tau), int(T), int(K))
            ctx.c_meta = (c.dtype, c.device)
            ctx.lam_is_tensor = torch.is_tensor(lam)
            ctx.save_for_backward(y)
            return x

        @staticmethod
        def backward(ctx, gx):
            (y,) = ctx.saved_tensors
            lam_f, tau, T, K = ctx.args
            dc = torch.empty(ctx.plan.n, dtype=torch.float32, device=y.device)
            dl = torch.empty(1, dtype=torch.float32, device=y.device)
            dy = torch.empty(ctx.plan.m, dtype=torch.float32, device=y.device)
            cs_grad(ctx.plan, y.detach().contiguous(), lam_f, tau, T, K, gx.contiguous().float(), dc, dl, dy)
            code = cs_status_sync(ctx.plan)
            ctx.plan.close()
            _check(code, "cs_grad")
            dlam = dl.reshape(()) if ctx.lam_is_tensor else None
            return dc.to(dtype=ctx.c_meta[0], device=ctx.c_meta[1]), dy, dlam, None, None, None, None

    return UnrolledISTA


def __getattr__(name):
    if name == "UnrolledISTA":
        cls = _make_unrolled_ista()
        globals()["UnrolledISTA"] = cls
        return cls
    raise AttributeError(name)


def cs_forward_direct(n: int, m: int, c, rows, x, y, stream=None):
    """y = A x by one O(n) dot product per kept row (context comparator);
    c float32 device (n,), rows int32 device (m,)."""
    rptr = _ptr(rows, dtype="torch.int32", numel=int(m))
    _check(_lib.cs_forward_direct(int(n), int(m), _ptr(c, numel=int(n)), rptr, _ptr(x, numel=int(n)),
                                  _ptr(y, numel=int(m)), _stream_handle(stream)),
           "cs_forward_direct")


def cs_profile_pass(plan: Plan, pass_id: int, reps: int = 1):
    _check(_lib.cs_profile_pass(plan.handle, int(pass_id), int(reps)), "cs_profile_pass")


def cs_circulant_apply_static(n: int, c, x, y, transpose: bool = False, stream=None):
    """y = C x (or C^T x) with no plan and no allocation (n <= 16384).
    c: float64 CUDA tensor (or device address) of at least n elements; x, y:
    float32 CUDA tensors of at least n elements.  Tensors of another dtype,
    on the host or too short are rejected here, before anything is launched."""
    n = int(n)
    cptr = _ptr(c, dtype="torch.float64", numel=n)
    _check(_lib.cs_circulant_apply_static(n, cptr, _ptr(x, numel=n), _ptr(y, numel=n), int(bool(transpose)),
                                          _stream_handle(stream)), "cs_circulant_apply_static")


class BatchPlan:
    """Owns a cs_batch_t: instances i = 0..count-1 with sizes n[i], m[i];
    their vectors are concatenated in instance order (offsets noff / moff)."""

    def __init__(self, handle: int, n, m):
        self.handle = handle
        self.n = np.asarray(n, dtype=np.int64)
        self.m = np.asarray(m, dtype=np.int64)
        self.noff = np.concatenate([[0], np.cumsum(self.n)[:-1]]).astype(np.int64)
        self.moff = np.concatenate([[0], np.cumsum(self.m)[:-1]]).astype(np.int64)
        self.count = len(self.n)

    def close(self):
        if self.handle:
            _lib.cs_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def cs_batch_plan(n, m, rows, c, stream=None) -> BatchPlan:
    """n, m: per-instance sizes; rows (int64) and c (float64): the instances'
    rows and generating vectors, concatenated."""
    n = np.ascontiguousarray(n, dtype=np.int64)
    m = np.ascontiguousarray(m, dtype=np.int64)
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    c = np.ascontiguousarray(c, dtype=np.float64)
    if n.shape != m.shape or rows.shape != (int(m.sum()),) or c.shape != (int(n.sum()),):
        raise ValueError("rows must hold sum(m) entries and c sum(n)")
    h = ctypes.c_void_p()
    code = _lib.cs_batch_plan(ctypes.byref(h), len(n), n.ctypes.data, m.ctypes.data, rows.ctypes.data,
                              c.ctypes.data, _stream_handle(stream))
    _check(code, "cs_batch_plan")
    return BatchPlan(h.value, n, m)


def cs_batch_destroy(batch: BatchPlan):
    batch.close()


def _host_f32(v, count: int) -> np.ndarray:
    a = np.ascontiguousarray(np.broadcast_to(np.asarray(v, dtype=np.float32), (count,)))
    return a


def cs_batch_ista(batch: BatchPlan, y, lam, tau, iters: int, x):
    """lam, tau: scalars or per-instance sequences (host)."""
    lam_h, tau_h = _host_f32(lam, batch.count), _host_f32(tau, batch.count)
    sn, sm = int(batch.n.sum()), int(batch.m.sum())
    _check(_lib.cs_batch_ista(batch.handle, _ptr(y, numel=sm), lam_h.ctypes.data, tau_h.ctypes.data, int(iters),
                              _ptr(x, numel=sn)), "cs_batch_ista")


def cs_batch_admm(batch: BatchPlan, y, lam, rho, iters: int, z):
    lam_h, rho_h = _host_f32(lam, batch.count), _host_f32(rho, batch.count)
    sn, sm = int(batch.n.sum()), int(batch.m.sum())
    _check(_lib.cs_batch_admm(batch.handle, _ptr(y, numel=sm), lam_h.ctypes.data, rho_h.ctypes.data, int(iters),
                              _ptr(z, numel=sn)), "cs_batch_admm")


def cs_batch_status_sync(batch: BatchPlan) -> int:
    return int(_lib.cs_batch_status_sync(batch.handle))


def cs_status_sync(plan: Plan) -> int:
    return int(_lib.cs_status_sync(plan.handle))


def raw_call(name: str, *args) -> int:
    """Call a C entry point with raw ctypes arguments and return its status
    (used by the C-ABI contract tests)."""
    return int(getattr(_lib, name)(*args))


def nan_to_none(v: float):
    return None if (v is None or (isinstance(v, float) and math.isnan(v))) else v
