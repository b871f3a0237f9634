"""Python binding of ``libafn.so`` (include/afn.h) -- argument marshalling only.

Every function here has the name of the C entry point it calls.  Arrays may
be numpy arrays (host memory) or torch tensors (host or CUDA memory); outputs
are returned in the same kind of memory as the main input.  All arithmetic
runs in the library's CUDA kernels: there is no fallback, and importing this
module raises if ``libafn.so`` has not been built (``__graft_entry__.build()``
or ``python -m paper_2304_05460_gb300.build``).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libafn.so")

AFN_OK, AFN_ERR_ARG, AFN_ERR_OOM, AFN_ERR_NOT_SPD, AFN_ERR_NO_CONVERGE = 0, 1, 2, 3, 4
AFN_ERR_TIMEOUT, AFN_ERR_CUDA, AFN_ERR_BUSY = 5, 6, 7
STATUS_NAMES = {0: "AFN_OK", 1: "AFN_ERR_ARG", 2: "AFN_ERR_OOM", 3: "AFN_ERR_NOT_SPD",
                4: "AFN_ERR_NO_CONVERGE", 5: "AFN_ERR_TIMEOUT", 6: "AFN_ERR_CUDA", 7: "AFN_ERR_BUSY"}
GAUSSIAN, MATERN32 = 0, 1
PREC_FP64, PREC_MIXED = 0, 1
LM_AUTO, LM_FPS, LM_UNIFORM = 0, 1, 2
RANK_FIXED, RANK_ESTIMATE = 0, 1


class AfnError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), msg))
        self.status = status


class afn_options(C.Structure):
    _fields_ = [("precision", C.c_int32), ("landmarks", C.c_int32), ("rank_mode", C.c_int32),
                ("rank_subsample", C.c_int32), ("fps_start", C.c_int64), ("seed", C.c_uint64),
                ("max_iter", C.c_int32), ("max_outer", C.c_int32), ("inner_tol", C.c_double),
                ("check_every", C.c_int32), ("profile", C.c_int32), ("stream", C.c_void_p)]


class afn_build_info(C.Structure):
    _fields_ = [("n", C.c_int64), ("nr", C.c_int64), ("k", C.c_int64), ("d", C.c_int32),
                ("w", C.c_int32), ("kernel", C.c_int32), ("precision", C.c_int32),
                ("rank_r", C.c_int64), ("rank_branch", C.c_int32), ("pad_", C.c_int32),
                ("l", C.c_double), ("mu", C.c_double), ("build_ms", C.c_double),
                ("device_bytes", C.c_int64)]


class afn_solve_info(C.Structure):
    _fields_ = [("iters", C.POINTER(C.c_int32)), ("relres", C.POINTER(C.c_double)),
                ("outer_steps", C.c_int32), ("converged", C.c_int32), ("solve_ms", C.c_double)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError("libafn.so is not built (%s); run __graft_entry__.build()" % LIB_PATH)
    lib = C.CDLL(LIB_PATH)
    P, i64, i32, dbl, u64 = C.c_void_p, C.c_int64, C.c_int32, C.c_double, C.c_uint64
    sig = {
        "afn_default_options": (None, [C.POINTER(afn_options)]),
        "afn_build": (i32, [P, i64, i32, i32, dbl, dbl, i32, i32, C.POINTER(afn_options),
                            C.POINTER(P)]),
        "afn_solve": (i32, [P, P, i32, dbl, P, C.POINTER(afn_solve_info)]),
        "afn_free": (None, [P]),
        "afn_last_error": (C.c_char_p, []),
        "afn_get_build_info": (i32, [P, C.POINTER(afn_build_info)]),
        "afn_get_perm": (i32, [P, P]),
        "afn_get_L": (i32, [P, P]),
        "afn_get_G": (i32, [P, P, P]),
        "afn_get_W": (i32, [P, P]),
        "afn_apply_precond": (i32, [P, P, i32, P]),
        "afn_get_kernel_stats": (i32, [P, C.c_char_p, C.POINTER(i64), C.POINTER(dbl)]),
        "afn_reset_kernel_stats": (i32, [P]),
        "afn_kernel_matvec": (i32, [P, i64, i32, i32, dbl, dbl, P, i32, P, i32, P]),
        "afn_fps": (i32, [P, i64, i32, i64, i64, P, P]),
        "afn_knn_pattern": (i32, [P, i64, i32, i32, P, P]),
        "afn_rank_estimate": (i32, [P, i64, i32, i32, dbl, dbl, i32, u64, i32, C.POINTER(i64),
                                    C.POINTER(i64), C.POINTER(i32), P]),
        "afn_launch_count": (i64, []),
        "afn_kernel_matvec_noalloc": (i32, [P, i64, i32, i32, dbl, dbl, P, i32, P, P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


_lib = _load()


def lib():
    return _lib


def last_error() -> str:
    return (_lib.afn_last_error() or b"").decode(errors="replace")


def _check(st):
    if st != AFN_OK:
        raise AfnError(st, last_error())


# ------------------------------------------------------------- marshalling --
def _is_torch(a):
    return type(a).__module__.startswith("torch")


def _ptr(a):
    """(pointer, keepalive) for a numpy array or torch tensor."""
    if _is_torch(a):
        if not a.is_contiguous():
            a = a.contiguous()
        return C.c_void_p(a.data_ptr()), a
    a = np.ascontiguousarray(a)
    return a.ctypes.data_as(C.c_void_p), a


def _f64_rowmajor(a):
    if _is_torch(a):
        import torch
        return a.to(torch.float64).contiguous()
    return np.ascontiguousarray(a, dtype=np.float64)


def _f64_colmajor(a):
    """n x m column-major float64 (as a contiguous m x n transpose buffer)."""
    if _is_torch(a):
        import torch
        t = a.to(torch.float64)
        if t.dim() == 1:
            return t.contiguous(), 1
        return t.t().contiguous(), t.shape[1]
    a = np.asarray(a, dtype=np.float64)
    if a.ndim == 1:
        return np.ascontiguousarray(a), 1
    return np.ascontiguousarray(a.T), a.shape[1]


def _empty_like_kind(ref, shape, dtype):
    if _is_torch(ref):
        import torch
        tdt = {np.float64: torch.float64, np.int64: torch.int64, np.int32: torch.int32}[dtype]
        return torch.empty(shape, dtype=tdt, device=ref.device)
    return np.empty(shape, dtype=dtype)


def _stream_ptr(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return C.c_void_p(stream)
    return C.c_void_p(stream.cuda_stream)


def options(**kw) -> afn_options:
    o = afn_options()
    _lib.afn_default_options(C.byref(o))
    for k, v in kw.items():
        if k == "stream":
            v = _stream_ptr(v)
        setattr(o, k, v)
    return o


# ------------------------------------------------------------------ handle --
class Handle:
    """Owns an ``afn_handle*``; frees it on ``afn_free`` / garbage collection."""

    def __init__(self, ptr, n, nrhs_kind):
        self.ptr = ptr
        self.n = n
        self._kind = nrhs_kind

    def __del__(self):
        try:
            afn_free(self)
        except Exception:
            pass

    @property
    def info(self) -> afn_build_info:
        return afn_get_build_info(self)


def afn_build(points, kernel, l, mu, k_max, fsai_nnz, opt: afn_options | None = None, **kw):
    """Alg. 2: landmarks, chol(K11 + mu I), W = L^{-1} K12, FSAI of the Schur complement."""
    X = _f64_rowmajor(points)
    n, d = int(X.shape[0]), int(X.shape[1])
    if opt is None:
        opt = options(**kw)
    px, keep = _ptr(X)
    h = C.c_void_p()
    _check(_lib.afn_build(px, n, d, int(kernel), float(l), float(mu), int(k_max), int(fsai_nnz),
                          C.byref(opt), C.byref(h)))
    return Handle(h, n, X)


def afn_free(h: Handle):
    if h is not None and h.ptr:
        _lib.afn_free(h.ptr)
        h.ptr = None


def afn_solve(h: Handle, rhs, tol):
    """PCG with the AFN preconditioner.  rhs: (n,) or (n, nrhs); returns
    (x, info) with info = dict(iters, relres, outer_steps, converged, solve_ms)."""
    B, nrhs = _f64_colmajor(rhs)
    if int(B.shape[-1]) != h.n:
        raise ValueError("rhs has %d rows, handle has n=%d" % (B.shape[-1], h.n))
    out = _empty_like_kind(B, tuple(B.shape), np.float64)
    its = (C.c_int32 * nrhs)()
    rel = (C.c_double * nrhs)()
    info = afn_solve_info(its, rel, 0, 0, 0.0)
    pb, kb = _ptr(B)
    po, ko = _ptr(out)
    st = _lib.afn_solve(h.ptr, pb, nrhs, float(tol), po, C.byref(info))
    if st not in (AFN_OK, AFN_ERR_NO_CONVERGE):
        _check(st)
    x = out.T if out.ndim == 2 else out
    res = dict(iters=np.array(its[:], dtype=np.int64), relres=np.array(rel[:]),
               outer_steps=info.outer_steps, converged=info.converged, solve_ms=info.solve_ms,
               status=st)
    return x, res


def afn_get_build_info(h: Handle) -> afn_build_info:
    bi = afn_build_info()
    _check(_lib.afn_get_build_info(h.ptr, C.byref(bi)))
    return bi


def afn_get_perm(h: Handle):
    out = np.empty(h.n, dtype=np.int64)
    _check(_lib.afn_get_perm(h.ptr, _ptr(out)[0]))
    return out


def afn_get_L(h: Handle):
    k = afn_get_build_info(h).k
    out = np.zeros((k, k), dtype=np.float64)
    if k:
        _check(_lib.afn_get_L(h.ptr, _ptr(out)[0]))
    return out


def afn_get_G(h: Handle):
    bi = afn_get_build_info(h)
    pat = np.full((bi.nr, bi.w), -1, dtype=np.int32)
    val = np.zeros((bi.nr, bi.w), dtype=np.float64)
    if bi.nr:
        _check(_lib.afn_get_G(h.ptr, _ptr(pat)[0], _ptr(val)[0]))
    return pat, val


def afn_get_W(h: Handle):
    bi = afn_get_build_info(h)
    out = np.zeros((bi.nr, bi.k), dtype=np.float64)
    if bi.nr and bi.k:
        _check(_lib.afn_get_W(h.ptr, _ptr(out)[0]))
    return out


def afn_apply_precond(h: Handle, r):
    """M^{-1} r (Alg. 3), FP64 handles; r in PERMUTED order, (n,) or (n, nrhs)."""
    R, nrhs = _f64_colmajor(r)
    out = np.empty(R.shape, dtype=np.float64)
    pr, kr = _ptr(R)
    _check(_lib.afn_apply_precond(h.ptr, pr, nrhs, _ptr(out)[0]))
    return out.T if out.ndim == 2 else out


def afn_get_kernel_stats(h: Handle, name: str):
    cnt = C.c_int64(0)
    ms = C.c_double(0.0)
    _check(_lib.afn_get_kernel_stats(h.ptr, name.encode(), C.byref(cnt), C.byref(ms)))
    return int(cnt.value), float(ms.value)


def afn_launch_count() -> int:
    """Kernels launched by libafn.so in this process so far."""
    return int(_lib.afn_launch_count())


def afn_reset_kernel_stats(h: Handle):
    _check(_lib.afn_reset_kernel_stats(h.ptr))


# ------------------------------------------------------- operator entries --
def afn_kernel_matvec(points, kernel, l, mu, p, precision=PREC_FP64, stream=None):
    """(K + mu I) p, matrix-free; p (n,) or (n, nrhs)."""
    X = _f64_rowmajor(points)
    n, d = int(X.shape[0]), int(X.shape[1])
    Pm, nrhs = _f64_colmajor(p)
    out = _empty_like_kind(Pm, tuple(Pm.shape), np.float64)
    px, kx = _ptr(X)
    pp, kp = _ptr(Pm)
    po, ko = _ptr(out)
    _check(_lib.afn_kernel_matvec(px, n, d, int(kernel), float(l), float(mu), pp, nrhs, po,
                                  int(precision), _stream_ptr(stream)))
    return out.T if out.ndim == 2 else out


def afn_kernel_matvec_noalloc(points, kernel, l, mu, p, q, stream=None):
    """FP64 (K + mu I) p into q without any device allocation.  points (n x d),
    p and q (n x nrhs) must be contiguous CUDA float64 tensors; p and q are
    passed as their transposes' storage (column-major n x nrhs)."""
    n, d = int(points.shape[0]), int(points.shape[1])
    nrhs = 1 if p.dim() == 1 else int(p.shape[0])
    _check(_lib.afn_kernel_matvec_noalloc(C.c_void_p(points.data_ptr()), n, d, int(kernel),
                                          float(l), float(mu), C.c_void_p(p.data_ptr()), nrhs,
                                          C.c_void_p(q.data_ptr()), _stream_ptr(stream)))
    return q


def afn_fps(points, k, start=0, stream=None):
    """Alg. 6: k landmark indices (start index, or -1 for the point nearest the centroid)."""
    X = _f64_rowmajor(points)
    n, d = int(X.shape[0]), int(X.shape[1])
    out = _empty_like_kind(X, (max(int(k), 1),), np.int64)
    px, kx = _ptr(X)
    po, ko = _ptr(out)
    _check(_lib.afn_fps(px, n, d, int(k), int(start), po, _stream_ptr(stream)))
    return out[: int(k)]


def afn_knn_pattern(xr, w, stream=None):
    """FSAI pattern (Sec. 3.1): nr x w int32, -1 padded, diagonal last."""
    X = _f64_rowmajor(xr)
    nr, d = int(X.shape[0]), int(X.shape[1])
    out = _empty_like_kind(X, (nr, int(w)), np.int32)
    px, kx = _ptr(X)
    po, ko = _ptr(out)
    _check(_lib.afn_knn_pattern(px, nr, d, int(w), po, _stream_ptr(stream)))
    return out


def afn_rank_estimate(points, kernel, l, mu, m=0, seed=0, k_max=4000, stream=None):
    """Alg. 4: returns (k, r, branch)."""
    X = _f64_rowmajor(points)
    n, d = int(X.shape[0]), int(X.shape[1])
    px, kx = _ptr(X)
    k = C.c_int64(0)
    r = C.c_int64(0)
    br = C.c_int32(0)
    _check(_lib.afn_rank_estimate(px, n, d, int(kernel), float(l), float(mu), int(m),
                                  C.c_uint64(int(seed) & (2**64 - 1)), int(k_max), C.byref(k),
                                  C.byref(r), C.byref(br), _stream_ptr(stream)))
    return int(k.value), int(r.value), int(br.value)
