"""Multi-shift conjugate gradient on NVIDIA GB300 (sm_103a).

Python binding of libmsc (include/msc.h). The functions named msc_* are the
C ABI one for one: they marshal arguments (numpy arrays, torch tensors or raw
pointers) and call the library; every step of the solve runs in the
library's CUDA kernels. There is no CPU fallback: if the library cannot be
loaded, every call raises.

Solves (A + sigma_s I) x_s = b for all shifts from one Krylov sequence
(CG-M, Algorithm 1, Sec. 2 of arXiv:1102.2143) for Hermitian positive-definite
A (`solve`, `solve_batched`), and by BiCGStab-M for non-Hermitian A
(`solve_nonherm`); `autograd.quad_form` differentiates the quadratic form
sum_s c_s phi^dag (A + sigma_s)^{-1} phi.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import inputs  # noqa: F401  (seeded synthetic inputs)

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libmsc.so")

MSC_OK = 0
MSC_ERR_ARG = 1
MSC_ERR_CUDA = 2
MSC_ERR_OOM = 3
MSC_ERR_NOT_HPD = 4
MSC_ERR_NONFINITE = 5
MSC_ERR_NOT_CONVERGED = 6
MSC_ERR_TIMEOUT = 7
MSC_ERR_UNSUPPORTED = 8
MSC_ERR_BREAKDOWN = 9

MSC_FP64 = 0
MSC_MIXED = 1
MSC_FP32 = 2
MSC_LINKS_FULL = 1
MSC_CHECK_HERMITIAN = 2

_lib = None
_lock = threading.Lock()


class MscError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {strerror(code)} (status {code})")


class msc_params(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("max_iter", ctypes.c_int), ("precision", ctypes.c_int),
                ("reliable_every", ctypes.c_int), ("freeze_converged", ctypes.c_int),
                ("refine", ctypes.c_int), ("reliable_delta", ctypes.c_double)]


class msc_info(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("iters", ctypes.c_int), ("refine_rounds", ctypes.c_int),
                ("refine_iters", ctypes.c_int), ("reliable_updates", ctypes.c_int),
                ("refine_reliable_updates", ctypes.c_int),
                ("kernel_launches", ctypes.c_int), ("seconds", ctypes.c_double),
                ("shift_iters", ctypes.POINTER(ctypes.c_int)),
                ("shift_refine_iters", ctypes.POINTER(ctypes.c_int)),
                ("true_rel_resid", ctypes.POINTER(ctypes.c_double)),
                ("op_ms", ctypes.c_double), ("rupdate_ms", ctypes.c_double),
                ("update_ms", ctypes.c_double), ("prof_samples", ctypes.c_int),
                ("prof_active", ctypes.c_double)]


class msc_problem(ctypes.Structure):
    _fields_ = [("op", ctypes.c_void_p), ("b", ctypes.c_void_p), ("nrhs", ctypes.c_int),
                ("sigma", ctypes.c_void_p), ("S", ctypes.c_int), ("x", ctypes.c_void_p),
                ("info", ctypes.POINTER(msc_info))]


class msc_tuning(ctypes.Structure):
    _fields_ = [("site_threads", ctypes.c_int), ("vec_threads", ctypes.c_int),
                ("vec_units", ctypes.c_int), ("tuned", ctypes.c_int), ("best_ms", ctypes.c_double)]


# exported symbols of include/msc.h with their ctypes signatures
_VP = ctypes.c_void_p
_I = ctypes.c_int
_I64 = ctypes.c_int64
_D = ctypes.c_double
SIGNATURES = {
    "msc_create": (_I, [ctypes.POINTER(_VP), _I, _VP]),
    "msc_destroy": (_I, [_VP]),
    "msc_set_stream": (_I, [_VP, _VP]),
    "msc_op_staggered": (_I, [_VP, ctypes.POINTER(_VP), _I, _VP, _VP, _D, ctypes.c_uint]),
    "msc_op_bsr": (_I, [_VP, ctypes.POINTER(_VP), _I64, _I, _VP, _VP, _VP, ctypes.c_uint]),
    "msc_op_bsr_size": (_I, [_VP, ctypes.POINTER(_I64), ctypes.POINTER(_I64), ctypes.POINTER(_I)]),
    "msc_staggered_export_bsr": (_I, [_VP, _VP, _VP, _VP, _VP]),
    "msc_op_size": (_I, [_VP, ctypes.POINTER(_I64)]),
    "msc_op_recon": (_I, [_VP, ctypes.POINTER(_I)]),
    "msc_op_apply": (_I, [_VP, _VP, _D, _VP, _VP, _I]),
    "msc_op_dslash": (_I, [_VP, _VP, _VP, _VP]),
    "msc_op_destroy": (_I, [_VP]),
    "msc_op_apply_noalloc": (_I, [_VP, _D, _VP, _VP, _VP]),
    "msc_params_default": (None, [ctypes.POINTER(msc_params)]),
    "msc_solve": (_I, [_VP, _VP, _VP, _I, _VP, _I, ctypes.POINTER(msc_params), _VP,
                       ctypes.POINTER(msc_info)]),
    "msc_solve_nonherm": (_I, [_VP, _VP, _VP, _I, _VP, _I, ctypes.POINTER(msc_params), _VP,
                       ctypes.POINTER(msc_info)]),
    "msc_solve_poly_rhs": (_I, [_VP, _VP, _VP, _VP, _I, _VP, _I, ctypes.POINTER(msc_params), _VP,
                                ctypes.POINTER(msc_info)]),
    "msc_solve_parity": (_I, [_VP, _VP, _I, _VP, _I, _VP, _I, ctypes.POINTER(msc_params), _VP,
                              ctypes.POINTER(msc_info)]),
    "msc_strerror": (ctypes.c_char_p, [_I]),
    "msc_quad_form": (_I, [_VP, _VP, _VP, _I, _VP, _VP, ctypes.POINTER(_D)]),
    "msc_quad_form_grad": (_I, [_VP, _VP, _I, _VP, _VP, _VP, _VP]),
    "msc_solve_batched": (_I, [_VP, _I, _VP, ctypes.POINTER(msc_params), _VP]),
}


def load(build_if_missing: bool = False):
    """Load libmsc.so (raises if it is missing: there is no fallback)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                if not build_if_missing:
                    raise ImportError(f"libmsc.so not built ({LIB_PATH}); run "
                                      "`python -c 'import __graft_entry__ as g; g.build()'`")
                from . import build as _b
                _b.build()
            L = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in SIGNATURES.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def strerror(code: int) -> str:
    try:
        return load().msc_strerror(int(code)).decode()
    except Exception:
        return f"status {code}"


def _check(code: int, where: str):
    if code != MSC_OK:
        raise MscError(code, where)


def _ptr(a):
    """Raw address of a numpy array, a torch tensor or an int."""
    if a is None:
        return None
    if isinstance(a, int):
        return a
    if isinstance(a, np.ndarray):
        assert a.flags["C_CONTIGUOUS"]
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        assert a.is_contiguous()
        return a.data_ptr()
    raise TypeError(type(a))


def _stream_handle(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


# ---------------------------------------------------------------------------
# C ABI, one for one
# ---------------------------------------------------------------------------

def msc_create(device: int = 0, stream=None) -> int:
    h = ctypes.c_void_p()
    _check(load().msc_create(ctypes.byref(h), int(device), _stream_handle(stream)), "msc_create")
    return h.value


def msc_destroy(ctx: int) -> None:
    _check(load().msc_destroy(ctx), "msc_destroy")


def msc_set_stream(ctx: int, stream) -> None:
    _check(load().msc_set_stream(ctx, _stream_handle(stream)), "msc_set_stream")


def msc_op_staggered(ctx: int, nc: int, dims, links, mass: float, flags: int = 0) -> int:
    d = (ctypes.c_int * 4)(*[int(v) for v in dims])
    h = ctypes.c_void_p()
    _check(load().msc_op_staggered(ctx, ctypes.byref(h), int(nc), ctypes.addressof(d), _ptr(links),
                                   float(mass), int(flags)), "msc_op_staggered")
    return h.value


def msc_op_bsr(ctx: int, nbr: int, bd: int, row_ptr, col_idx, vals, flags: int = 0) -> int:
    h = ctypes.c_void_p()
    _check(load().msc_op_bsr(ctx, ctypes.byref(h), int(nbr), int(bd), _ptr(row_ptr), _ptr(col_idx),
                             _ptr(vals), int(flags)), "msc_op_bsr")
    return h.value


def msc_op_bsr_size(op: int):
    nbr, nnzb, bd = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int()
    _check(load().msc_op_bsr_size(op, ctypes.byref(nbr), ctypes.byref(nnzb), ctypes.byref(bd)),
           "msc_op_bsr_size")
    return nbr.value, nnzb.value, bd.value


def msc_staggered_export_bsr(ctx: int, op: int, row_ptr, col_idx, vals) -> None:
    _check(load().msc_staggered_export_bsr(ctx, op, _ptr(row_ptr), _ptr(col_idx), _ptr(vals)),
           "msc_staggered_export_bsr")


def msc_op_size(op: int) -> int:
    n = ctypes.c_int64()
    _check(load().msc_op_size(op, ctypes.byref(n)), "msc_op_size")
    return n.value


def msc_op_recon(op: int) -> int:
    r = ctypes.c_int()
    _check(load().msc_op_recon(op, ctypes.byref(r)), "msc_op_recon")
    return r.value


def msc_op_apply(ctx: int, op: int, sigma: float, x, out, precision: int = MSC_FP64) -> None:
    _check(load().msc_op_apply(ctx, op, float(sigma), _ptr(x), _ptr(out), int(precision)),
           "msc_op_apply")


def msc_op_dslash(ctx: int, op: int, x, out) -> None:
    _check(load().msc_op_dslash(ctx, op, _ptr(x), _ptr(out)), "msc_op_dslash")


def msc_op_apply_noalloc(op: int, sigma: float, x, out, stream=None) -> None:
    """out = (A + sigma) x without any allocation (device pointers; queued on
    `stream`, returns without waiting).

    The library takes no length here and stages nothing, so a torch tensor
    must be a contiguous complex128 CUDA tensor of exactly n entries (n the
    operator's size), x and out on the same device; anything else raises
    before the call. Raw integer addresses are passed through unchecked."""
    tensors = [a for a in (x, out) if hasattr(a, "data_ptr")]
    if tensors:
        import torch
        n = msc_op_size(op)
        for a in tensors:
            if a.dtype != torch.complex128 or not a.is_contiguous() or not a.is_cuda:
                raise ValueError("msc_op_apply_noalloc: x and out must be contiguous complex128 "
                                 "CUDA tensors")
            if a.numel() != n:
                raise ValueError(f"msc_op_apply_noalloc: {a.numel()} entries, the operator has {n}")
        if len({a.device for a in tensors}) > 1:
            raise ValueError("msc_op_apply_noalloc: x and out are on different devices")
    _check(load().msc_op_apply_noalloc(op, float(sigma), _ptr(x), _ptr(out), _stream_handle(stream)),
           "msc_op_apply_noalloc")


def msc_op_destroy(op: int) -> None:
    _check(load().msc_op_destroy(op), "msc_op_destroy")


def msc_quad_form(ctx: int, op: int, phi, S: int, coef, x) -> float:
    """S = sum_s c_s Re(phi^dag x_s) on the device (x: [S][n] solved x_s)."""
    cf = np.ascontiguousarray(coef, dtype=np.float64)
    v = ctypes.c_double()
    _check(load().msc_quad_form(ctx, op, _ptr(phi), int(S), _ptr(cf), _ptr(x), ctypes.byref(v)),
           "msc_quad_form")
    return v.value


def msc_quad_form_grad(ctx: int, op: int, S: int, coef, x, dphi=None, dU=None) -> None:
    """dphi = 2 sum_s c_s x_s and the link force dU (see include/msc.h)."""
    cf = np.ascontiguousarray(coef, dtype=np.float64)
    _check(load().msc_quad_form_grad(ctx, op, int(S), _ptr(cf), _ptr(x), _ptr(dphi), _ptr(dU)),
           "msc_quad_form_grad")


_contexts = {}


def default_context(device: int = 0) -> int:
    """A context per device for the convenience and autograd layers."""
    with _lock:
        h = _contexts.get(device)
    if h is None:
        h = msc_create(device, None)
        with _lock:
            _contexts[device] = h
    return h


def msc_params_default() -> msc_params:
    p = msc_params()
    load().msc_params_default(ctypes.byref(p))
    return p


def msc_solve(ctx: int, op: int, b, nrhs: int, sigma, S: int, params: msc_params, x,
              info: msc_info | None = None) -> int:
    """Raw call; returns the status (MSC_ERR_NOT_CONVERGED is not raised)."""
    return load().msc_solve(ctx, op, _ptr(b), int(nrhs), _ptr(sigma), int(S),
                            ctypes.byref(params), _ptr(x),
                            ctypes.byref(info) if info is not None else None)


def msc_solve_nonherm(ctx: int, op: int, b, nrhs: int, sigma, S: int, params: msc_params, x,
                      info: msc_info | None = None) -> int:
    """Raw call of the BiCGStab-M solve; returns the status."""
    return load().msc_solve_nonherm(ctx, op, _ptr(b), int(nrhs), _ptr(sigma), int(S),
                                    ctypes.byref(params), _ptr(x),
                                    ctypes.byref(info) if info is not None else None)


def msc_solve_poly_rhs(ctx: int, op: int, b, sigma, S: int, coef, deg: int, params: msc_params, x,
                       info: msc_info | None = None) -> int:
    """Raw call of the polynomial right-hand-side solve; returns the status."""
    return load().msc_solve_poly_rhs(ctx, op, _ptr(b), _ptr(sigma), int(S), _ptr(coef), int(deg),
                                     ctypes.byref(params), _ptr(x),
                                     ctypes.byref(info) if info is not None else None)


def msc_solve_parity(ctx: int, op: int, parity: int, b, nrhs: int, sigma, S: int, params: msc_params, x,
                     info: msc_info | None = None) -> int:
    """Raw call of the single-parity solve; returns the status."""
    return load().msc_solve_parity(ctx, op, int(parity), _ptr(b), int(nrhs), _ptr(sigma), int(S),
                                   ctypes.byref(params), _ptr(x),
                                   ctypes.byref(info) if info is not None else None)


# ---------------------------------------------------------------------------
# convenience layer (still only marshalling)
# ---------------------------------------------------------------------------

class SolveInfo:
    def __init__(self, info: msc_info, shift_iters, refine_iters, resid):
        for name, _ in msc_info._fields_:
            if name not in ("shift_iters", "shift_refine_iters", "true_rel_resid"):
                setattr(self, name, getattr(info, name))
        self.shift_iters = shift_iters
        self.shift_refine_iters = refine_iters
        self.true_rel_resid = resid


def solve(ctx: int, op: int, b, sigma, x=None, tol=1e-10, precision=MSC_MIXED, max_iter=100000,
          reliable_every=50, freeze=True, refine=4, raise_on_error=True):
    """Solve for all shifts. `b`: [nrhs][n] (or [n]) complex128 numpy array or
    torch tensor, host or device; `x` (optional) receives [nrhs][S][n].
    Returns (x, SolveInfo)."""
    sig = np.ascontiguousarray(sigma, dtype=np.float64)
    S = int(sig.shape[0])
    squeeze = False
    if hasattr(b, "data_ptr"):
        import torch
        if b.dim() == 1:
            b = b.unsqueeze(0)
            squeeze = True
        b = b.contiguous()
        nrhs, n = b.shape
        if x is None:
            x = torch.empty((nrhs, S, n), dtype=torch.complex128, device=b.device)
    else:
        b = np.ascontiguousarray(b, dtype=np.complex128)
        if b.ndim == 1:
            b = b[None, :]
            squeeze = True
        nrhs, n = b.shape
        if x is None:
            x = np.empty((nrhs, S, n), dtype=np.complex128)
    p = msc_params_default()
    p.tol, p.max_iter, p.precision = float(tol), int(max_iter), int(precision)
    p.reliable_every, p.freeze_converged, p.refine = int(reliable_every), int(bool(freeze)), int(refine)
    it = np.zeros(nrhs * S, dtype=np.int32)
    rit = np.zeros(nrhs * S, dtype=np.int32)
    rho = np.zeros(nrhs * S, dtype=np.float64)
    info = msc_info()
    info.shift_iters = it.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
    info.shift_refine_iters = rit.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
    info.true_rel_resid = rho.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    st = msc_solve(ctx, op, b, nrhs, sig, S, p, x, info)
    if st != MSC_OK and (raise_on_error and st != MSC_ERR_NOT_CONVERGED):
        raise MscError(st, "msc_solve")
    res = SolveInfo(info, it.reshape(nrhs, S), rit.reshape(nrhs, S), rho.reshape(nrhs, S))
    if squeeze:
        x = x[0]
    return x, res


def solve_parity(ctx: int, op: int, parity: int, b, sigma, x=None, tol=1e-10, precision=MSC_MIXED,
                 max_iter=100000, reliable_every=50, freeze=True, refine=4, raise_on_error=True):
    """Shifted family for a source on the sites of one parity (0 even, 1
    odd) of a staggered operator. `b`: [nrhs][V/2*nc] (or [V/2*nc]) complex128,
    the parity's sites in site order (site x at index x // 2); `x` (optional)
    receives [nrhs][S][V/2*nc]. Returns (x, SolveInfo)."""
    sig = np.ascontiguousarray(sigma, dtype=np.float64)
    S = int(sig.shape[0])
    squeeze = False
    if hasattr(b, "data_ptr"):
        import torch
        if b.dim() == 1:
            b = b.unsqueeze(0)
            squeeze = True
        b = b.contiguous()
        nrhs, n = b.shape
        if x is None:
            x = torch.empty((nrhs, S, n), dtype=torch.complex128, device=b.device)
    else:
        b = np.ascontiguousarray(b, dtype=np.complex128)
        if b.ndim == 1:
            b = b[None, :]
            squeeze = True
        nrhs, n = b.shape
        if x is None:
            x = np.empty((nrhs, S, n), dtype=np.complex128)
    p = msc_params_default()
    p.tol, p.max_iter, p.precision = float(tol), int(max_iter), int(precision)
    p.reliable_every, p.freeze_converged, p.refine = int(reliable_every), int(bool(freeze)), int(refine)
    it = np.zeros(nrhs * S, dtype=np.int32)
    rit = np.zeros(nrhs * S, dtype=np.int32)
    rho = np.zeros(nrhs * S, dtype=np.float64)
    info = msc_info()
    info.shift_iters = it.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
    info.shift_refine_iters = rit.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
    info.true_rel_resid = rho.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    st = msc_solve_parity(ctx, op, parity, b, nrhs, sig, S, p, x, info)
    if st != MSC_OK and (raise_on_error and st != MSC_ERR_NOT_CONVERGED):
        raise MscError(st, "msc_solve_parity")
    res = SolveInfo(info, it.reshape(nrhs, S), rit.reshape(nrhs, S), rho.reshape(nrhs, S))
    if squeeze:
        x = x[0]
    return x, res


def solve_poly_rhs(ctx: int, op: int, b, sigma, coef, x=None, tol=1e-10, precision=MSC_MIXED,
                   max_iter=100000, reliable_every=50, refine=4, raise_on_error=True):
    """(A + sigma_s) x_s = q_s(A) b for every shift, q_s(t) = sum_k coef[s][k] t^k.
    `b`: [n] complex128 (numpy or torch, host or device); `coef`: [S][deg+1]
    real; `x` (optional) receives [S][n]. Returns (x, SolveInfo); the
    residuals in the info are relative to |q_s(A) b|."""
    sig = np.ascontiguousarray(sigma, dtype=np.float64)
    S = int(sig.shape[0])
    cf = np.ascontiguousarray(coef, dtype=np.float64).reshape(S, -1)
    deg = cf.shape[1] - 1
    if hasattr(b, "data_ptr"):
        import torch
        b = b.reshape(-1).contiguous()
        n = b.shape[0]
        if x is None:
            x = torch.empty((S, n), dtype=torch.complex128, device=b.device)
    else:
        b = np.ascontiguousarray(b, dtype=np.complex128).reshape(-1)
        n = b.shape[0]
        if x is None:
            x = np.empty((S, n), dtype=np.complex128)
    p = msc_params_default()
    p.tol, p.max_iter, p.precision = float(tol), int(max_iter), int(precision)
    p.reliable_every, p.refine = int(reliable_every), int(refine)
    it = np.zeros(S, dtype=np.int32)
    rit = np.zeros(S, dtype=np.int32)
    rho = np.zeros(S, dtype=np.float64)
    info = msc_info()
    info.shift_iters = it.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
    info.shift_refine_iters = rit.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
    info.true_rel_resid = rho.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    st = msc_solve_poly_rhs(ctx, op, b, sig, S, cf, deg, p, x, info)
    if st != MSC_OK and (raise_on_error and st != MSC_ERR_NOT_CONVERGED):
        raise MscError(st, "msc_solve_poly_rhs")
    return x, SolveInfo(info, it, rit, rho)


def solve_nonherm(ctx: int, op: int, b, sigma, x=None, tol=1e-10, max_iter=100000, freeze=True,
                  raise_on_error=True):
    """Non-Hermitian shifted family by BiCGStab-M (FP64, block-CSR operator).
    `b`: [nrhs][n] (or [n]) complex128, numpy or torch, host or device; `x`
    (optional) receives [nrhs][S][n]. Returns (x, SolveInfo)."""
    sig = np.ascontiguousarray(sigma, dtype=np.float64)
    S = int(sig.shape[0])
    squeeze = False
    if hasattr(b, "data_ptr"):
        import torch
        if b.dim() == 1:
            b = b.unsqueeze(0)
            squeeze = True
        b = b.contiguous()
        nrhs, n = b.shape
        if x is None:
            x = torch.empty((nrhs, S, n), dtype=torch.complex128, device=b.device)
    else:
        b = np.ascontiguousarray(b, dtype=np.complex128)
        if b.ndim == 1:
            b = b[None, :]
            squeeze = True
        nrhs, n = b.shape
        if x is None:
            x = np.empty((nrhs, S, n), dtype=np.complex128)
    p = msc_params_default()
    p.tol, p.max_iter, p.precision = float(tol), int(max_iter), MSC_FP64
    p.freeze_converged = int(bool(freeze))
    it = np.zeros(nrhs * S, dtype=np.int32)
    rit = np.zeros(nrhs * S, dtype=np.int32)
    rho = np.zeros(nrhs * S, dtype=np.float64)
    info = msc_info()
    info.shift_iters = it.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
    info.shift_refine_iters = rit.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
    info.true_rel_resid = rho.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    st = msc_solve_nonherm(ctx, op, b, nrhs, sig, S, p, x, info)
    if st != MSC_OK and (raise_on_error and st != MSC_ERR_NOT_CONVERGED):
        raise MscError(st, "msc_solve_nonherm")
    res = SolveInfo(info, it.reshape(nrhs, S), rit.reshape(nrhs, S), rho.reshape(nrhs, S))
    if squeeze:
        x = x[0]
    return x, res


def msc_solve_batched(ctx: int, problems, params: msc_params, tuning: msc_tuning | None = None) -> int:
    """Raw call on a ctypes array of msc_problem; returns the status."""
    arr = (msc_problem * len(problems))(*problems)
    return load().msc_solve_batched(ctx, len(problems), ctypes.addressof(arr), ctypes.byref(params),
                                    ctypes.addressof(tuning) if tuning is not None else None)


def solve_batched(ctx: int, items, tol=1e-10, precision=MSC_MIXED, max_iter=100000,
                  reliable_every=50, freeze=True, refine=4, raise_on_error=True):
    """Solve many staggered problems together. `items`: list of (op, b, sigma)
    with b [nrhs][n] complex128 (numpy or torch, host or device). Returns
    (list of x [nrhs][S][n], list of SolveInfo, msc_tuning)."""
    probs, keep, outs, infos = [], [], [], []
    for op, b, sigma in items:
        sig = np.ascontiguousarray(sigma, dtype=np.float64)
        S = int(sig.shape[0])
        if hasattr(b, "data_ptr"):
            import torch
            if b.dim() == 1:
                b = b.unsqueeze(0)
            b = b.contiguous()
            nrhs, n = b.shape
            x = torch.empty((nrhs, S, n), dtype=torch.complex128, device=b.device)
        else:
            b = np.ascontiguousarray(b, dtype=np.complex128)
            if b.ndim == 1:
                b = b[None, :]
            nrhs, n = b.shape
            x = np.empty((nrhs, S, n), dtype=np.complex128)
        it = np.zeros(nrhs * S, dtype=np.int32)
        rit = np.zeros(nrhs * S, dtype=np.int32)
        rho = np.zeros(nrhs * S, dtype=np.float64)
        info = msc_info()
        info.shift_iters = it.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
        info.shift_refine_iters = rit.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
        info.true_rel_resid = rho.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        keep.append((b, sig, it, rit, rho, info))
        probs.append(msc_problem(op, _ptr(b), nrhs, sig.ctypes.data, S, _ptr(x), ctypes.pointer(info)))
        outs.append(x)
    p = msc_params_default()
    p.tol, p.max_iter, p.precision = float(tol), int(max_iter), int(precision)
    p.reliable_every, p.freeze_converged, p.refine = int(reliable_every), int(bool(freeze)), int(refine)
    tun = msc_tuning()
    st = msc_solve_batched(ctx, probs, p, tun)
    if st != MSC_OK and raise_on_error and st != MSC_ERR_NOT_CONVERGED:
        raise MscError(st, "msc_solve_batched")
    for (b, sig, it, rit, rho, info), x in zip(keep, outs):
        nrhs = x.shape[0]
        S = x.shape[1]
        infos.append(SolveInfo(info, it.reshape(nrhs, S), rit.reshape(nrhs, S), rho.reshape(nrhs, S)))
    return outs, infos, tun
