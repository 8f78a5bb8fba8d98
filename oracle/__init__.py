"""FP64 CPU oracle for the shifted-family solve (A + sigma_i I) x_i = b.

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's CPU
baseline leg use it; the library in `paper_1102_2143_gb300` never imports,
links or runs anything here, and this package imports nothing from it.

The arithmetic lives in `msc_oracle.c` (plain loops, double precision); this
module compiles it with gcc and exposes it to numpy through ctypes. Every
function follows the paper's statement of the problem (eq. linprob, Sec. 2)
and CG-M (Algorithm 1, Sec. 2, with the readings listed in the C file), and
BiCGStab-M for non-Hermitian families (named in Sec. 1 and Sec. 3, not
printed; its recurrences are derived in the C file's header).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "msc_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lib = None
_lock = threading.Lock()

STATUS = {0: "ok", 1: "bad argument", 4: "not HPD", 5: "non-finite", 6: "not converged",
          7: "breakdown"}


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/_build/liboracle.so (gcc, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB_PATH)
            dp = ctypes.POINTER(ctypes.c_double)
            ip = ctypes.POINTER(ctypes.c_int)
            i64p = ctypes.POINTER(ctypes.c_int64)
            i32p = ctypes.POINTER(ctypes.c_int32)
            L.orc_num_threads.restype = ctypes.c_int
            L.orc_set_threads.argtypes = [ctypes.c_int]
            L.orc_cgm_staggered.argtypes = [ctypes.c_int, ip, dp, ctypes.c_double, dp, ctypes.c_int,
                                            dp, ctypes.c_double, ctypes.c_int, ctypes.c_int, dp, ip,
                                            ip, dp, dp]
            L.orc_cgm_bsr.argtypes = [ctypes.c_long, ctypes.c_int, i64p, i32p, dp, dp, ctypes.c_int,
                                      dp, ctypes.c_double, ctypes.c_int, ctypes.c_int, dp, ip, ip,
                                      dp, dp]
            L.orc_cg_staggered.argtypes = [ctypes.c_int, ip, dp, ctypes.c_double, dp,
                                           ctypes.c_double, ctypes.c_double, ctypes.c_int, dp, ip]
            L.orc_cg_bsr.argtypes = [ctypes.c_long, ctypes.c_int, i64p, i32p, dp, dp,
                                     ctypes.c_double, ctypes.c_double, ctypes.c_int, dp, ip]
            L.orc_dslash_c.argtypes = [ctypes.c_int, ip, dp, dp, dp]
            L.orc_staggered_apply_c.argtypes = [ctypes.c_int, ip, dp, ctypes.c_double,
                                                ctypes.c_double, dp, dp]
            L.orc_bsr_apply_c.argtypes = [ctypes.c_long, ctypes.c_int, i64p, i32p, dp,
                                          ctypes.c_double, dp, dp]
            L.orc_true_residual_staggered.argtypes = [ctypes.c_int, ip, dp, ctypes.c_double, dp,
                                                      ctypes.c_int, dp, dp, dp]
            L.orc_link_force.argtypes = [ctypes.c_int, ip, dp, ctypes.c_int, dp, dp, dp]
            L.orc_bicgstabm_bsr.argtypes = [ctypes.c_long, ctypes.c_int, i64p, i32p, dp, dp,
                                            ctypes.c_int, dp, ctypes.c_double, ctypes.c_int,
                                            ctypes.c_int, dp, ip, ip, dp, dp]
            L.orc_bicgstabm_dirac.argtypes = [ctypes.c_int, ip, dp, ctypes.c_double, dp, ctypes.c_int,
                                              dp, ctypes.c_double, ctypes.c_int, ctypes.c_int, dp, ip,
                                              ip, dp, dp]
            L.orc_dirac_apply_c.argtypes = [ctypes.c_int, ip, dp, ctypes.c_double, ctypes.c_double,
                                            dp, dp]
            for f in ("orc_cgm_staggered", "orc_cgm_bsr", "orc_cg_staggered", "orc_cg_bsr",
                      "orc_bicgstabm_bsr", "orc_bicgstabm_dirac"):
                getattr(L, f).restype = ctypes.c_int
            _lib = L
    return _lib


def _c128(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.complex128)


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def _dims(dims) -> np.ndarray:
    d = np.asarray(dims, dtype=np.int32)
    assert d.shape == (4,)
    return d


def num_threads() -> int:
    return lib().orc_num_threads()


def set_threads(n: int) -> None:
    lib().orc_set_threads(int(n))


# ----------------------------------------------------------------------------
# Operators
# ----------------------------------------------------------------------------

def dslash(links, dims, nc, v) -> np.ndarray:
    """D v for the staggered operator."""
    U, v = _c128(links), _c128(v)
    out = np.empty_like(v)
    d = _dims(dims)
    lib().orc_dslash_c(nc, _ip(d), _dp(U), _dp(v), _dp(out))
    return out


def staggered_apply(links, dims, nc, mass, v, sigma: float = 0.0) -> np.ndarray:
    """(A + sigma) v with A = m^2 - D^2."""
    U, v = _c128(links), _c128(v)
    out = np.empty_like(v)
    d = _dims(dims)
    lib().orc_staggered_apply_c(nc, _ip(d), _dp(U), float(mass), float(sigma), _dp(v), _dp(out))
    return out


def bsr_apply(row_ptr, col_idx, vals, v, sigma: float = 0.0) -> np.ndarray:
    rp = np.ascontiguousarray(row_ptr, dtype=np.int64)
    ci = np.ascontiguousarray(col_idx, dtype=np.int32)
    va = _c128(vals)
    v = _c128(v)
    bd = va.shape[-1]
    nbr = rp.shape[0] - 1
    out = np.empty_like(v)
    lib().orc_bsr_apply_c(nbr, bd, rp.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                          ci.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), _dp(va),
                          float(sigma), _dp(v), _dp(out))
    return out


# ----------------------------------------------------------------------------
# Solvers
# ----------------------------------------------------------------------------

class CGMResult:
    def __init__(self, x, conv_iter, iters, status, zeta, r):
        self.x = x                  # [S][n]
        self.conv_iter = conv_iter  # [S]
        self.iters = iters
        self.status = status
        self.zeta = zeta            # [S] final zeta_0 per shift
        self.r = r                  # final unshifted residual


def cgm_staggered(links, dims, nc, mass, b, sigma, tol, max_iter=100000, freeze=True) -> CGMResult:
    """CG-M (Algorithm 1) on the staggered operator, all shifts from one Krylov sequence."""
    U, b = _c128(links), _c128(b)
    sig = np.ascontiguousarray(sigma, dtype=np.float64)
    S, n = sig.shape[0], b.shape[0]
    x = np.zeros((S, n), dtype=np.complex128)
    conv = np.zeros(S, dtype=np.int32)
    it = np.zeros(1, dtype=np.int32)
    zeta = np.zeros(S, dtype=np.float64)
    r = np.zeros(n, dtype=np.complex128)
    d = _dims(dims)
    st = lib().orc_cgm_staggered(nc, _ip(d), _dp(U), float(mass), _dp(b), S, _dp(sig), float(tol),
                                 int(max_iter), int(bool(freeze)), _dp(x), _ip(conv), _ip(it),
                                 _dp(zeta), _dp(r))
    return CGMResult(x, conv, int(it[0]), st, zeta, r)


def cgm_bsr(row_ptr, col_idx, vals, b, sigma, tol, max_iter=100000, freeze=True) -> CGMResult:
    """CG-M (Algorithm 1) on a generic block-CSR operator."""
    rp = np.ascontiguousarray(row_ptr, dtype=np.int64)
    ci = np.ascontiguousarray(col_idx, dtype=np.int32)
    va, b = _c128(vals), _c128(b)
    sig = np.ascontiguousarray(sigma, dtype=np.float64)
    S, n = sig.shape[0], b.shape[0]
    x = np.zeros((S, n), dtype=np.complex128)
    conv = np.zeros(S, dtype=np.int32)
    it = np.zeros(1, dtype=np.int32)
    zeta = np.zeros(S, dtype=np.float64)
    r = np.zeros(n, dtype=np.complex128)
    st = lib().orc_cgm_bsr(rp.shape[0] - 1, va.shape[-1],
                           rp.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                           ci.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), _dp(va), _dp(b), S,
                           _dp(sig), float(tol), int(max_iter), int(bool(freeze)), _dp(x), _ip(conv),
                           _ip(it), _dp(zeta), _dp(r))
    return CGMResult(x, conv, int(it[0]), st, zeta, r)


class BiCGStabMResult:
    def __init__(self, x, conv_iter, iters, status, c, r):
        self.x = x                  # [S][n]
        self.conv_iter = conv_iter  # [S]
        self.iters = iters
        self.status = status
        self.c = c                  # [S] complex zeta_sigma / T_sigma at exit
        self.r = r                  # final seed residual


def bicgstabm_bsr(row_ptr, col_idx, vals, b, sigma, tol, max_iter=100000, freeze=True) -> BiCGStabMResult:
    """BiCGStab-M on a generic (non-Hermitian) block-CSR operator: all
    (A + sigma_s) x_s = b from one BiCGStab sequence on A."""
    rp = np.ascontiguousarray(row_ptr, dtype=np.int64)
    ci = np.ascontiguousarray(col_idx, dtype=np.int32)
    va, b = _c128(vals), _c128(b)
    sig = np.ascontiguousarray(sigma, dtype=np.float64)
    S, n = sig.shape[0], b.shape[0]
    x = np.zeros((S, n), dtype=np.complex128)
    conv = np.zeros(S, dtype=np.int32)
    it = np.zeros(1, dtype=np.int32)
    c = np.zeros(S, dtype=np.complex128)
    r = np.zeros(n, dtype=np.complex128)
    st = lib().orc_bicgstabm_bsr(rp.shape[0] - 1, va.shape[-1],
                                 rp.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                 ci.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), _dp(va), _dp(b), S,
                                 _dp(sig), float(tol), int(max_iter), int(bool(freeze)), _dp(x),
                                 _ip(conv), _ip(it), _dp(c), _dp(r))
    return BiCGStabMResult(x, conv, int(it[0]), st, c, r)


def bicgstabm_dirac(links, dims, nc, mass, b, sigma, tol, max_iter=100000, freeze=True) -> BiCGStabMResult:
    """BiCGStab-M on the staggered Dirac operator M = m + D: the multi-mass
    family (m + sigma_s + D) x_s = b."""
    U, b = _c128(links), _c128(b)
    sig = np.ascontiguousarray(sigma, dtype=np.float64)
    S, n = sig.shape[0], b.shape[0]
    x = np.zeros((S, n), dtype=np.complex128)
    conv = np.zeros(S, dtype=np.int32)
    it = np.zeros(1, dtype=np.int32)
    c = np.zeros(S, dtype=np.complex128)
    r = np.zeros(n, dtype=np.complex128)
    d = _dims(dims)
    st = lib().orc_bicgstabm_dirac(nc, _ip(d), _dp(U), float(mass), _dp(b), S, _dp(sig), float(tol),
                                   int(max_iter), int(bool(freeze)), _dp(x), _ip(conv), _ip(it),
                                   _dp(c), _dp(r))
    return BiCGStabMResult(x, conv, int(it[0]), st, c, r)


def dirac_apply(links, dims, nc, mass, v, sigma: float = 0.0) -> np.ndarray:
    """(m + sigma + D) v, the staggered Dirac operator."""
    U, v = _c128(links), _c128(v)
    out = np.zeros_like(v)
    d = _dims(dims)
    lib().orc_dirac_apply_c(nc, _ip(d), _dp(U), float(mass), float(sigma), _dp(v), _dp(out))
    return out


def cg_staggered(links, dims, nc, mass, b, sigma, tol, max_iter=100000):
    """Textbook CG on (A + sigma) x = b from x = 0. Returns (x, iters, status)."""
    U, b = _c128(links), _c128(b)
    x = np.zeros_like(b)
    it = np.zeros(1, dtype=np.int32)
    d = _dims(dims)
    st = lib().orc_cg_staggered(nc, _ip(d), _dp(U), float(mass), _dp(b), float(sigma), float(tol),
                                int(max_iter), _dp(x), _ip(it))
    return x, int(it[0]), st


def cg_bsr(row_ptr, col_idx, vals, b, sigma, tol, max_iter=100000):
    rp = np.ascontiguousarray(row_ptr, dtype=np.int64)
    ci = np.ascontiguousarray(col_idx, dtype=np.int32)
    va, b = _c128(vals), _c128(b)
    x = np.zeros_like(b)
    it = np.zeros(1, dtype=np.int32)
    st = lib().orc_cg_bsr(rp.shape[0] - 1, va.shape[-1],
                          rp.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                          ci.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), _dp(va), _dp(b),
                          float(sigma), float(tol), int(max_iter), _dp(x), _ip(it))
    return x, int(it[0]), st


def true_residual_staggered(links, dims, nc, mass, b, sigma, x) -> np.ndarray:
    """rho_s = |b - (A + sigma_s) x_s| / |b| in FP64, x: [S][n]."""
    U, b, x = _c128(links), _c128(b), _c128(x)
    sig = np.ascontiguousarray(sigma, dtype=np.float64)
    rho = np.zeros(sig.shape[0], dtype=np.float64)
    d = _dims(dims)
    lib().orc_true_residual_staggered(nc, _ip(d), _dp(U), float(mass), _dp(b), sig.shape[0],
                                      _dp(sig), _dp(x), _dp(rho))
    return rho


def link_force(links, dims, nc, c, x) -> np.ndarray:
    """dS/dU for S = sum_s c_s Re(phi^dagger x_s); x: [S][n] solved x_s."""
    U, x = _c128(links), _c128(x)
    cc = np.ascontiguousarray(c, dtype=np.float64)
    G = np.zeros_like(U)
    d = _dims(dims)
    lib().orc_link_force(nc, _ip(d), _dp(U), cc.shape[0], _dp(cc), _dp(x), _dp(G))
    return G


def quad_form(b, x, c) -> float:
    """S = sum_s c_s Re(phi^dagger x_s)."""
    return float(sum(float(c[s]) * np.vdot(b, x[s]).real for s in range(len(c))))


# ----------------------------------------------------------------------------
# Different right-hand side per shift (Sec. 5, eq. linprobgen), for
# right-hand sides of polynomial form b_s = q_s(A) b. Written from the
# definition: each b_s is formed by Horner's rule with the FP64 operator and
# each shift is solved on its own by textbook CG.
# ----------------------------------------------------------------------------

def poly_apply_staggered(links, dims, nc, mass, coef, b) -> np.ndarray:
    """q(A) b with q(t) = sum_k coef[k] t^k (coef[0] the constant term), by
    Horner's rule: v = coef[d] b, then v = A v + coef[k] b for k = d-1 .. 0."""
    coef = np.asarray(coef, dtype=np.float64)
    b = _c128(b)
    v = coef[-1] * b
    for a in coef[-2::-1]:
        v = staggered_apply(links, dims, nc, mass, v) + a * b
    return v


def solve_poly_rhs_staggered(links, dims, nc, mass, b, sigma, coef, tol, max_iter=100000):
    """x_s = (A + sigma_s)^{-1} q_s(A) b for every shift s (coef: [S][deg+1]),
    each by textbook CG from x = 0 to |b_s - (A + sigma_s) x_s| <= tol |b_s|.
    Returns (x [S][n], b_s [S][n])."""
    sig = np.asarray(sigma, dtype=np.float64)
    coef = np.asarray(coef, dtype=np.float64).reshape(sig.shape[0], -1)
    xs, bs = [], []
    for s in range(sig.shape[0]):
        bq = poly_apply_staggered(links, dims, nc, mass, coef[s], b)
        if np.linalg.norm(bq) == 0.0:
            x = np.zeros_like(bq)
        else:
            x, _, st = cg_staggered(links, dims, nc, mass, bq, sig[s], tol, max_iter)
            if st != 0:
                raise RuntimeError(f"oracle CG for shift {s}: {STATUS.get(st, st)}")
        xs.append(x)
        bs.append(bq)
    return np.array(xs), np.array(bs)
