"""ctypes binding of the C-ABI in ``include/pp.h`` (argument marshalling only).

Every function here has the name of the C entry point it calls and does no
arithmetic of the method: the polynomial build, apply and Arnoldi iteration
all run in ``libpp.so``.  Importing this module loads the library and raises
if it has not been built (``__graft_entry__.build()``); there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpp.so")

PP_OK, PP_ENOTCONV, PP_EBREAKDOWN, PP_EAGAIN = 0, 1, 2, 3
PP_EINVAL, PP_ENOMEM, PP_ECUDA, PP_ETIMEOUT, PP_ENUMERIC = -1, -2, -3, -4, -5
PP_FP64, PP_FP32, PP_FP32_BF16 = 0, 1, 2
PP_FMT_AUTO, PP_FMT_CSR, PP_FMT_SELL, PP_FMT_DIA = 0, 1, 2, 3
PP_TARGET_SM, PP_TARGET_SR = 0, 1
PP_RESTART_RITZ, PP_RESTART_HARMONIC = 0, 1


class pp_opts(C.Structure):
    _fields_ = [("precision", C.c_int), ("format", C.c_int), ("target", C.c_int), ("sigma", C.c_double),
                ("add_roots", C.c_int), ("max_cycles", C.c_int), ("refine_steps", C.c_int),
                ("sell_c", C.c_int), ("sell_sigma", C.c_int), ("sell_index", C.c_int), ("sell_loop", C.c_int),
                ("stream", C.c_void_p), ("restart", C.c_int), ("balance", C.c_int), ("dia_loop", C.c_int)]


class pp_stats(C.Structure):
    _fields_ = [("cycles", C.c_int64), ("mvps", C.c_int64), ("dots", C.c_int64), ("vops", C.c_int64),
                ("kernel_launches", C.c_int64), ("converged", C.c_int32), ("nconv", C.c_int32),
                ("t_total", C.c_double), ("t_apply", C.c_double), ("t_orth", C.c_double),
                ("t_restart", C.c_double), ("max_resid", C.c_double), ("fp64_cycles", C.c_int64)]

    def to_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class PPError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"pp status {status}: {msg}")
        self.status = status


_P = C.c_void_p
_D = C.POINTER(C.c_double)
_I = C.POINTER(C.c_int)
_I64 = C.POINTER(C.c_int64)

_SIGS = {
    "pp_opts_default": (None, [C.POINTER(pp_opts)]),
    "pp_last_error": (C.c_char_p, []),
    "pp_create": (C.c_int, [C.POINTER(_P), C.c_int64, _I64, C.POINTER(C.c_int32), _D, C.POINTER(pp_opts)]),
    "pp_destroy": (None, [_P]),
    "pp_trim": (C.c_int, [_P]),
    "pp_matrix_info": (C.c_int, [_P, _D, _D]),
    "pp_csr_info": (C.c_int, [C.c_int64, _I64, C.POINTER(C.c_int32), _D, _D, _D]),
    "pp_csr_balance": (C.c_int, [C.c_int64, _I64, C.POINTER(C.c_int32), _D, _D, _D]),
    "pp_balance_info": (C.c_int, [_P, _I, _D]),
    "pp_debug_stall_sweeps": (C.c_int, [_P, C.c_int]),
    "pp_format_info": (C.c_int, [_P, _I, _I, _I, _I, _I, _I64]),
    "pp_launch_count": (C.c_int64, [_P]),
    "pp_build_poly": (C.c_int, [_P, C.c_int, _D, C.POINTER(_P)]),
    "pp_build_poly2": (C.c_int, [_P, C.c_int, C.c_int, _D, C.POINTER(_P)]),
    "pp_build_poly_two": (C.c_int, [_P, C.c_int, _D, _D, C.POINTER(_P)]),
    "pp_build_poly_damped": (C.c_int, [_P, C.c_int, _D, C.c_int, C.c_int, C.c_int, C.POINTER(_P), _I, _I, _I]),
    "pp_poly_from_roots": (C.c_int, [_P, C.c_int, _D, _D, C.POINTER(_P)]),
    "pp_poly2_from_roots": (C.c_int, [_P, C.c_int, _D, _D, C.c_int, _D, _D, C.POINTER(_P)]),
    "pp_poly_roots": (C.c_int, [_P, _D, _D, C.c_int, _I]),
    "pp_poly_inner_roots": (C.c_int, [_P, _D, _D, C.c_int, _I]),
    "pp_poly_info": (C.c_int, [_P, _I, _I]),
    "pp_poly_counts": (C.c_int, [_P, _I64, _I64, _I64]),
    "pp_poly_destroy": (None, [_P]),
    "pp_apply": (C.c_int, [_P, _P, _P]),
    "pp_apply_host": (C.c_int, [_P, _D, _D]),
    "pp_eigs": (C.c_int, [_P, _P, C.c_int, C.c_int, C.c_int, C.c_double, _D, _D, _D, _D, _D, _I,
                          C.POINTER(pp_stats)]),
    "pp_orthogonalize": (C.c_int, [_P, _P, C.c_int64, C.c_int, _P, _P, _D]),
    "pp_orthogonalize_noalloc": (C.c_int, [C.c_int64, _P, C.c_int64, C.c_int, _P, _P, _P, _P]),
    "pp_batch_create": (C.c_int, [C.POINTER(_P), C.c_int, _I64, C.POINTER(_I64), C.POINTER(C.POINTER(C.c_int32)),
                                  C.POINTER(_D), C.POINTER(pp_opts)]),
    "pp_batch_solve": (C.c_int, [_P, _I, C.POINTER(_D), C.POINTER(_D), C.c_int, C.c_int, C.c_int, C.c_double,
                                 C.POINTER(_D), C.POINTER(_D), C.POINTER(_D), C.POINTER(_D), _I, C.POINTER(pp_stats)]),
    "pp_batch_launch_count": (C.c_int64, [_P]),
    "pp_batch_destroy": (None, [_P]),
    "pp_server_create": (C.c_int, [C.POINTER(_P), C.POINTER(pp_opts), C.c_int64, C.c_int, C.c_int]),
    "pp_server_submit": (C.c_int, [_P, C.c_int64, _I64, C.POINTER(C.c_int32), _D, C.c_int, C.c_int, C.c_int,
                                   C.c_int, C.c_double, _D, _D, _I64]),
    "pp_server_step": (C.c_int, [_P, _I, _I]),
    "pp_server_result": (C.c_int, [_P, C.c_int64, _D, _D, _D, _D, _I, C.POINTER(pp_stats), _D]),
    "pp_server_launch_count": (C.c_int64, [_P]),
    "pp_server_request_bytes": (C.c_int64, [_P, C.c_int64, C.c_int64, C.c_int, C.c_int]),
    "pp_server_destroy": (None, [_P]),
    "pp_dense_eig": (C.c_int, [C.c_int, _D, C.c_int, _D, _D, _D, C.c_int]),
    "pp_harmonic_ritz": (C.c_int, [C.c_int, _D, C.c_int, _D, _D]),
    "pp_leja_order": (C.c_int, [C.c_int, _D, _D, _D, _D]),
    "pp_add_stability_roots": (C.c_int, [C.c_int, _D, _D, C.c_int, _D, _D, _I]),
    "pp_measure_fp64_rate": (C.c_int, [_P, _D]),
    "pp_restart_basis": (C.c_int, [C.c_int, _D, C.c_int, C.c_int, C.c_double, C.c_int, _D, _D, _I, _D, _D]),
}


def _load() -> C.CDLL:
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with __graft_entry__.build() "
                          "(there is no CPU fallback)")
    lib = C.CDLL(LIB_PATH)
    for name, (res, args) in _SIGS.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


LIB = _load()


def exported_symbols() -> list[str]:
    """Names of the C entry points this binding declares (all exported by libpp.so)."""
    return list(_SIGS)


def _check(status: int, allow=(PP_OK,)) -> int:
    if status in allow:
        return status
    raise PPError(status, LIB.pp_last_error().decode(errors="replace"))


def _dp(a: np.ndarray):
    return a.ctypes.data_as(_D)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _vec_in(a, n: int):
    """(keep-alive object, double*) for an input vector of n FP64 values: a CUDA
    array (anything with __cuda_array_interface__, e.g. a torch tensor on the
    GPU: float64, contiguous) is passed as its device pointer, anything else as
    a host copy."""
    cai = getattr(a, "__cuda_array_interface__", None)
    if cai is not None:
        if cai["typestr"] != "<f8" or tuple(cai["shape"]) not in ((n,), (n, 1)) or cai.get("strides") not in (None, (8,)):
            raise ValueError("device start vector: need n contiguous float64 values")
        return a, C.cast(C.c_void_p(int(cai["data"][0])), _D)
    h = _f64(a)
    if h.size != n:
        raise ValueError(f"start vector: need {n} values, got {h.size}")
    return h, _dp(h)


# ---------------------------------------------------------------------------
# Handles
# ---------------------------------------------------------------------------
class Context:
    """Owner of a pp_ctx handle (the uploaded matrix and its device scratch)."""

    def __init__(self, handle: int, n: int, precision: int):
        self.handle = C.c_void_p(handle)
        self.n = n
        self.precision = precision

    def close(self):
        if self.handle:
            LIB.pp_destroy(self.handle)
            self.handle = C.c_void_p(0)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Poly:
    """Owner of a pp_poly handle; keeps its context alive."""

    def __init__(self, handle: int, ctx: Context, status: int):
        self.handle = C.c_void_p(handle)
        self.ctx = ctx
        self.status = status

    def close(self):
        if self.handle:
            LIB.pp_poly_destroy(self.handle)
            self.handle = C.c_void_p(0)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def default_opts(**kw) -> pp_opts:
    o = pp_opts()
    LIB.pp_opts_default(C.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def pp_create(A, **opts) -> Context:
    """A: object with n, rowptr (int64), colind (int32), vals (float64)."""
    o = default_opts(**opts)
    rp = np.ascontiguousarray(A.rowptr, dtype=np.int64)
    ci = np.ascontiguousarray(A.colind, dtype=np.int32)
    va = _f64(A.vals)
    h = C.c_void_p()
    _check(LIB.pp_create(C.byref(h), int(A.n), rp.ctypes.data_as(_I64), ci.ctypes.data_as(C.POINTER(C.c_int32)),
                         _dp(va), C.byref(o)))
    return Context(h.value, int(A.n), o.precision)


def pp_balance_info(ctx: Context) -> tuple[bool, float]:
    """(balanced, log of the scaling range) of a context (pp_opts.balance)."""
    b, r = C.c_int(), C.c_double()
    _check(LIB.pp_balance_info(ctx.handle, C.byref(b), C.byref(r)))
    return bool(b.value), r.value


def pp_csr_info(A) -> tuple[float, float]:
    """(||A||_1, the smallest-real-part shift) of a host CSR matrix, as pp_create computes them."""
    rp = np.ascontiguousarray(A.rowptr, dtype=np.int64)
    ci = np.ascontiguousarray(A.colind, dtype=np.int32)
    va = _f64(A.vals)
    a, s = C.c_double(), C.c_double()
    _check(LIB.pp_csr_info(int(A.n), rp.ctypes.data_as(_I64), ci.ctypes.data_as(C.POINTER(C.c_int32)), _dp(va),
                           C.byref(a), C.byref(s)))
    return a.value, s.value


def pp_csr_balance(A) -> tuple[np.ndarray, float]:
    """(d, log range) of the symmetrising diagonal similarity of a host CSR matrix, as
    pp_create(balance=1) computes it; PPError (PP_EINVAL) when none exists."""
    rp = np.ascontiguousarray(A.rowptr, dtype=np.int64)
    ci = np.ascontiguousarray(A.colind, dtype=np.int32)
    va = _f64(A.vals)
    d = np.empty(int(A.n))
    r = C.c_double()
    _check(LIB.pp_csr_balance(int(A.n), rp.ctypes.data_as(_I64), ci.ctypes.data_as(C.POINTER(C.c_int32)), _dp(va),
                              _dp(d), C.byref(r)))
    return d, r.value


def pp_matrix_info(ctx: Context) -> tuple[float, float]:
    a, s = C.c_double(), C.c_double()
    _check(LIB.pp_matrix_info(ctx.handle, C.byref(a), C.byref(s)))
    return a.value, s.value


def pp_format_info(ctx: Context) -> dict:
    """Device format of A: fmt, chunk height, index bits, block size, row loop, stored entries."""
    f, c, ib, t, w = C.c_int(), C.c_int(), C.c_int(), C.c_int(), C.c_int()
    st = C.c_int64()
    _check(LIB.pp_format_info(ctx.handle, C.byref(f), C.byref(c), C.byref(ib), C.byref(t), C.byref(w),
                              C.byref(st)))
    return {"fmt": f.value, "chunk": c.value, "index_bits": ib.value, "threads": t.value, "row_loop": w.value,
            "stored": st.value}


def pp_debug_stall_sweeps(ctx: Context, count: int) -> None:
    """Test support: the next `count` staged CGS2 steps issue no copies (their waits run out)."""
    _check(LIB.pp_debug_stall_sweeps(ctx.handle, int(count)))


def pp_trim(ctx: Context) -> None:
    """Free the device workspace the context keeps between calls."""
    _check(LIB.pp_trim(ctx.handle))


def pp_launch_count(ctx: Context) -> int:
    return int(LIB.pp_launch_count(ctx.handle))


def pp_build_poly(ctx: Context, d: int, b) -> Poly:
    """GMRES polynomial of degree d from b (host array or float64 CUDA array)."""
    b, bp = _vec_in(b, ctx.n)
    h = C.c_void_p()
    st = _check(LIB.pp_build_poly(ctx.handle, int(d), bp, C.byref(h)), allow=(PP_OK, PP_EBREAKDOWN))
    return Poly(h.value, ctx, st)


def pp_build_poly_two(ctx: Context, d: int, b1, b2) -> Poly:
    """Polynomial from two starting vectors (Section 5 box)."""
    (b1, p1), (b2, p2) = _vec_in(b1, ctx.n), _vec_in(b2, ctx.n)
    h = C.c_void_p()
    st = _check(LIB.pp_build_poly_two(ctx.handle, int(d), p1, p2, C.byref(h)),
                allow=(PP_OK, PP_EBREAKDOWN))
    return Poly(h.value, ctx, st)


def pp_build_poly_damped(ctx: Context, d: int, b, m: int, k: int, nev: int) -> tuple[Poly, dict]:
    """Damping heuristic (Section 6.3 box); returns the polynomial and degree / damped / ideal."""
    b, bp = _vec_in(b, ctx.n)
    h = C.c_void_p()
    deg, dmp, ide = C.c_int(), C.c_int(), C.c_int()
    st = _check(LIB.pp_build_poly_damped(ctx.handle, int(d), bp, int(m), int(k), int(nev), C.byref(h),
                                         C.byref(deg), C.byref(dmp), C.byref(ide)), allow=(PP_OK, PP_EBREAKDOWN))
    return Poly(h.value, ctx, st), {"degree": deg.value, "damped": bool(dmp.value), "ideal": bool(ide.value)}


def pp_build_poly2(ctx: Context, d1: int, d2: int, b) -> Poly:
    b, bp = _vec_in(b, ctx.n)
    h = C.c_void_p()
    st = _check(LIB.pp_build_poly2(ctx.handle, int(d1), int(d2), bp, C.byref(h)), allow=(PP_OK, PP_EBREAKDOWN))
    return Poly(h.value, ctx, st)


def pp_poly_from_roots(ctx: Context, roots) -> Poly:
    r = np.asarray(roots, dtype=complex)
    re, im = _f64(r.real), _f64(r.imag)
    h = C.c_void_p()
    _check(LIB.pp_poly_from_roots(ctx.handle, int(r.size), _dp(re), _dp(im), C.byref(h)))
    return Poly(h.value, ctx, PP_OK)


def pp_poly2_from_roots(ctx: Context, inner_roots, outer_roots) -> Poly:
    """Double polynomial pi_2(tau(A)), tau = 1 - pi_1, with the given root lists (Section 8)."""
    r1 = np.asarray(inner_roots, dtype=complex)
    r2 = np.asarray(outer_roots, dtype=complex)
    re1, im1, re2, im2 = _f64(r1.real), _f64(r1.imag), _f64(r2.real), _f64(r2.imag)
    h = C.c_void_p()
    _check(LIB.pp_poly2_from_roots(ctx.handle, int(r1.size), _dp(re1), _dp(im1), int(r2.size), _dp(re2), _dp(im2),
                                   C.byref(h)))
    return Poly(h.value, ctx, PP_OK)


def _roots(fn, p: Poly) -> np.ndarray:
    cnt = C.c_int()
    _check(fn(p.handle, None, None, 0, C.byref(cnt)))
    re = np.zeros(max(cnt.value, 1))
    im = np.zeros(max(cnt.value, 1))
    _check(fn(p.handle, _dp(re), _dp(im), cnt.value, C.byref(cnt)))
    return (re + 1j * im)[: cnt.value]


def pp_poly_roots(p: Poly) -> np.ndarray:
    return _roots(LIB.pp_poly_roots, p)


def pp_poly_inner_roots(p: Poly) -> np.ndarray:
    return _roots(LIB.pp_poly_inner_roots, p)


def pp_poly_info(p: Poly) -> tuple[int, int]:
    d, a = C.c_int(), C.c_int()
    _check(LIB.pp_poly_info(p.handle, C.byref(d), C.byref(a)))
    return d.value, a.value


def pp_poly_counts(p: Poly) -> dict:
    m, d, v = C.c_int64(), C.c_int64(), C.c_int64()
    _check(LIB.pp_poly_counts(p.handle, C.byref(m), C.byref(d), C.byref(v)))
    return dict(mvps=m.value, dots=d.value, vops=v.value)


def pp_apply(p: Poly, x_dev: int, y_dev: int) -> None:
    """y = pi(A) x on device pointers (context storage type, asynchronous on its stream)."""
    _check(LIB.pp_apply(p.handle, C.c_void_p(int(x_dev)), C.c_void_p(int(y_dev))))


def pp_apply_host(p: Poly, x) -> np.ndarray:
    x = _f64(x)
    y = np.empty_like(x)
    _check(LIB.pp_apply_host(p.handle, _dp(x), _dp(y)))
    return y


def pp_orthogonalize(ctx: Context, V_dev: int, ldv: int, j: int, w_dev: int, v_dev: int) -> np.ndarray:
    """CGS2 of w against V[:, :j] on the device; returns h (j coefficients, then the norm)."""
    h = np.zeros(j + 1)
    _check(LIB.pp_orthogonalize(ctx.handle, C.c_void_p(int(V_dev)), int(ldv), int(j), C.c_void_p(int(w_dev)),
                                C.c_void_p(int(v_dev)), _dp(h)))
    return h


def pp_orthogonalize_noalloc(n: int, V_dev: int, ldv: int, j: int, w_dev: int, v_dev: int, h_dev: int,
                             stream: int = 0) -> None:
    """The CGS2 step without any allocation: every pointer is the caller's device memory."""
    _check(LIB.pp_orthogonalize_noalloc(int(n), C.c_void_p(int(V_dev)), int(ldv), int(j), C.c_void_p(int(w_dev)),
                                        C.c_void_p(int(v_dev)), C.c_void_p(int(h_dev)), C.c_void_p(int(stream))))


@dataclass
class EigsResult:
    lam: np.ndarray
    X: np.ndarray | None
    resid: np.ndarray
    status: int
    stats: dict


def pp_eigs(ctx: Context, p: Poly | None, nev: int, m: int, k: int, rtol: float, v0=None,
            want_vectors: bool = True, X_out: np.ndarray | None = None) -> EigsResult:
    """X_out: optional float64 C-contiguous (nev+1, n) host array the vectors are written
    into (e.g. pinned memory reused across calls); the result's X is a view of it."""
    n = ctx.n
    cap = nev + 1
    lre, lim, res = np.zeros(cap), np.zeros(cap), np.zeros(cap)
    if X_out is not None:
        if X_out.dtype != np.float64 or X_out.shape != (cap, n) or not X_out.flags.c_contiguous:
            raise ValueError("X_out must be a C-contiguous float64 array of shape (nev + 1, n)")
        X = X_out
    else:
        X = np.empty((cap, n)) if want_vectors else None  # slot-major: the library writes column s at X[s]
    v0a, v0p = _vec_in(v0, n) if v0 is not None else (None, None)
    nout = C.c_int()
    st = pp_stats()
    status = _check(LIB.pp_eigs(ctx.handle, p.handle if p is not None else None, int(nev), int(m), int(k),
                                float(rtol), v0p, _dp(lre), _dp(lim),
                                _dp(X) if X is not None else None, _dp(res), C.byref(nout), C.byref(st)),
                    allow=(PP_OK, PP_ENOTCONV))
    k_ = nout.value
    # X[:, j] is slot j's vector: a transposed view of the slot-major block (no copy)
    return EigsResult(lre[:k_] + 1j * lim[:k_], X[:k_].T if X is not None else None, res[:k_], status,
                      st.to_dict())


# ---------------------------------------------------------------------------
# Batching
# ---------------------------------------------------------------------------
class Batch:
    """Owner of a pp_batch handle (count instances)."""

    def __init__(self, handle: int, ns: list[int]):
        self.handle = C.c_void_p(handle)
        self.ns = ns

    def close(self):
        if self.handle:
            LIB.pp_batch_destroy(self.handle)
            self.handle = C.c_void_p(0)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def pp_batch_create(mats, **opts) -> Batch:
    o = default_opts(**opts)
    cnt = len(mats)
    keep = []
    ns = (C.c_int64 * cnt)(*[int(A.n) for A in mats])
    rps = (_I64 * cnt)()
    cis = (C.POINTER(C.c_int32) * cnt)()
    vas = (_D * cnt)()
    for i, A in enumerate(mats):
        rp = np.ascontiguousarray(A.rowptr, dtype=np.int64)
        ci = np.ascontiguousarray(A.colind, dtype=np.int32)
        va = _f64(A.vals)
        keep += [rp, ci, va]
        rps[i] = rp.ctypes.data_as(_I64)
        cis[i] = ci.ctypes.data_as(C.POINTER(C.c_int32))
        vas[i] = _dp(va)
    h = C.c_void_p()
    _check(LIB.pp_batch_create(C.byref(h), cnt, ns, rps, cis, vas, C.byref(o)))
    return Batch(h.value, [int(A.n) for A in mats])


def pp_batch_launch_count(b: Batch) -> int:
    return int(LIB.pp_batch_launch_count(b.handle))


def pp_batch_solve(b: Batch, d, bvecs, v0s, nev: int, m: int, k: int, rtol: float,
                   want_vectors: bool = True) -> tuple[int, list[EigsResult]]:
    cnt = len(b.ns)
    cap = nev + 1
    keep = []

    def arr(vs):
        a = (_D * cnt)()
        for i, v in enumerate(vs):
            if v is None:
                a[i] = _D()
            else:
                v = _f64(v)
                keep.append(v)
                a[i] = _dp(v)
        return a

    dd = (C.c_int * cnt)(*[int(x) for x in d])
    lre = [np.zeros(cap) for _ in range(cnt)]
    lim = [np.zeros(cap) for _ in range(cnt)]
    res = [np.zeros(cap) for _ in range(cnt)]
    Xs = [np.zeros((cap, n)) for n in b.ns] if want_vectors else None
    nout = (C.c_int * cnt)()
    stats = (pp_stats * cnt)()
    Xa = (_D * cnt)(*[_dp(x) for x in Xs]) if want_vectors else None
    status = _check(LIB.pp_batch_solve(b.handle, dd, arr(bvecs), arr(v0s) if v0s is not None else None, int(nev),
                                       int(m), int(k), float(rtol), (_D * cnt)(*[_dp(x) for x in lre]),
                                       (_D * cnt)(*[_dp(x) for x in lim]), Xa, (_D * cnt)(*[_dp(x) for x in res]),
                                       nout, stats), allow=(PP_OK, PP_ENOTCONV))
    out = []
    for i in range(cnt):
        k_ = nout[i]
        st = stats[i].to_dict()
        out.append(EigsResult(lre[i][:k_] + 1j * lim[i][:k_], Xs[i][:k_].T if want_vectors else None,
                              res[i][:k_], PP_OK if st["converged"] else PP_ENOTCONV, st))
    return status, out


# ---------------------------------------------------------------------------
# Serving
# ---------------------------------------------------------------------------
class Server:
    """Owner of a pp_server handle; remembers n and nev per request id."""

    def __init__(self, handle: int, keep_vectors: bool):
        self.handle = C.c_void_p(handle)
        self.keep_vectors = keep_vectors
        self.meta: dict[int, tuple[int, int]] = {}

    def close(self):
        if self.handle:
            LIB.pp_server_destroy(self.handle)
            self.handle = C.c_void_p(0)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def pp_server_create(mem_budget: int = 0, max_active: int = 0, keep_vectors: bool = False, **opts) -> Server:
    o = default_opts(**opts)
    h = C.c_void_p()
    _check(LIB.pp_server_create(C.byref(h), C.byref(o), int(mem_budget), int(max_active), int(keep_vectors)))
    return Server(h.value, keep_vectors)


def pp_server_submit(s: Server, A, d: int, nev: int, m: int, k: int, rtol: float, b, v0=None) -> int:
    rp = np.ascontiguousarray(A.rowptr, dtype=np.int64)
    ci = np.ascontiguousarray(A.colind, dtype=np.int32)
    va = _f64(A.vals)
    b = _f64(b)
    v0a = _f64(v0) if v0 is not None else None
    rid = C.c_int64()
    _check(LIB.pp_server_submit(s.handle, int(A.n), rp.ctypes.data_as(_I64), ci.ctypes.data_as(C.POINTER(C.c_int32)),
                                _dp(va), int(d), int(nev), int(m), int(k), float(rtol), _dp(b),
                                _dp(v0a) if v0a is not None else None, C.byref(rid)))
    s.meta[rid.value] = (int(A.n), int(nev))
    return rid.value


def pp_server_step(s: Server) -> tuple[int, int]:
    a, q = C.c_int(), C.c_int()
    _check(LIB.pp_server_step(s.handle, C.byref(a), C.byref(q)))
    return a.value, q.value


def pp_server_result(s: Server, rid: int):
    """None while pending, else (EigsResult, latency seconds)."""
    n, nev = s.meta[rid]
    cap = nev + 1
    lre, lim, res = np.zeros(cap), np.zeros(cap), np.zeros(cap)
    X = np.zeros((cap, n)) if s.keep_vectors else None
    nout, st, lat = C.c_int(), pp_stats(), C.c_double()
    status = LIB.pp_server_result(s.handle, int(rid), _dp(lre), _dp(lim), _dp(X) if X is not None else None,
                                  _dp(res), C.byref(nout), C.byref(st), C.byref(lat))
    if status == PP_EAGAIN:
        return None
    _check(status, allow=(PP_OK, PP_ENOTCONV))
    k_ = nout.value
    del s.meta[rid]
    return EigsResult(lre[:k_] + 1j * lim[:k_], X[:k_].T if X is not None else None, res[:k_], status,
                      st.to_dict()), lat.value


def pp_server_request_bytes(s: Server, n: int, nnz: int, m: int, nev: int) -> int:
    return int(LIB.pp_server_request_bytes(s.handle, int(n), int(nnz), int(m), int(nev)))


def pp_server_launch_count(s: Server) -> int:
    return int(LIB.pp_server_launch_count(s.handle))


# ---------------------------------------------------------------------------
# Host FP64 dense steps (no GPU needed)
# ---------------------------------------------------------------------------
def pp_dense_eig(A: np.ndarray, vectors: bool = True):
    A = np.asfortranarray(A, dtype=np.float64)
    n = A.shape[0]
    wr, wi = np.zeros(n), np.zeros(n)
    V = np.zeros((n, n), order="F") if vectors else None
    _check(LIB.pp_dense_eig(n, A.ctypes.data_as(_D), n, _dp(wr), _dp(wi),
                            V.ctypes.data_as(_D) if V is not None else None, n))
    return wr + 1j * wi, V


def pp_harmonic_ritz(H: np.ndarray) -> np.ndarray:
    H = np.asfortranarray(H, dtype=np.float64)
    d = H.shape[1]
    re, im = np.zeros(d), np.zeros(d)
    _check(LIB.pp_harmonic_ritz(d, H.ctypes.data_as(_D), H.shape[0], _dp(re), _dp(im)))
    return re + 1j * im


def pp_leja_order(roots) -> np.ndarray:
    r = np.asarray(roots, dtype=complex)
    re, im = _f64(r.real), _f64(r.imag)
    ore, oim = np.zeros(r.size), np.zeros(r.size)
    _check(LIB.pp_leja_order(r.size, _dp(re), _dp(im), _dp(ore), _dp(oim)))
    return ore + 1j * oim


def pp_add_stability_roots(roots) -> np.ndarray:
    r = np.asarray(roots, dtype=complex)
    re, im = _f64(r.real), _f64(r.imag)
    cap = 8 * r.size + 8
    ore, oim = np.zeros(cap), np.zeros(cap)
    cnt = C.c_int()
    _check(LIB.pp_add_stability_roots(r.size, _dp(re), _dp(im), cap, _dp(ore), _dp(oim), C.byref(cnt)))
    return (ore + 1j * oim)[: cnt.value]


def pp_restart_basis(H: np.ndarray, k: int, target: float, harmonic: bool = False):
    """Host step of one thick restart (see include/pp.h): returns (Q or P, Hn, kk, ordered values)."""
    H = np.asfortranarray(H, dtype=np.float64)
    m = H.shape[1]
    Q = np.zeros((m + 1) * (m + 1))
    Hn = np.zeros((m + 1, m), order="F")
    kk = C.c_int()
    re, im = np.zeros(m), np.zeros(m)
    _check(LIB.pp_restart_basis(int(m), H.ctypes.data_as(_D), int(m + 1), int(k), float(target), int(bool(harmonic)),
                                _dp(Q), Hn.ctypes.data_as(_D), C.byref(kk), _dp(re), _dp(im)))
    kv = kk.value
    rows, cols = (m + 1, kv + 1) if harmonic else (m, kv)
    return Q[: rows * cols].reshape((rows, cols), order="F"), Hn, kv, re + 1j * im


def pp_measure_fp64_rate(stream: int = 0) -> float:
    """Measured FP64 FMA throughput of the current GPU in flop/s."""
    r = C.c_double()
    _check(LIB.pp_measure_fp64_rate(C.c_void_p(int(stream)), C.byref(r)))
    return r.value
