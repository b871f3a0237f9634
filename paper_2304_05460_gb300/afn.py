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
PREC_FP64, PREC_MIXED, PREC_DF, PREC_AUTO = 0, 1, 2, 3
PRECOND_AFN, PRECOND_NYSTROM, PRECOND_AUTO = 0, 1, 2
MATVEC_DF = PREC_DF        # afn_kernel_matvec: FP64-accurate double-float
MATVEC_DF_TC, MATVEC_DF_CC = 4, 5   # ... with the sum over j on the tensor cores / FP32 pipes
LM_AUTO, LM_FPS, LM_UNIFORM = 0, 1, 2
RANK_FIXED, RANK_ESTIMATE = 0, 1
FACTORS_FP32, FACTORS_FP64 = 0, 1
KRYLOV_FP32, KRYLOV_FP64, KRYLOV_RESTART, KRYLOV_FP64_OPERATOR = 0, 1, 2, 3


class AfnError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), msg))
        self.status = status


class afn_options(C.Structure):
    _fields_ = [("precision", C.c_int32), ("landmarks", C.c_int32), ("rank_mode", C.c_int32),
                ("rank_subsample", C.c_int32), ("fps_start", C.c_int64), ("seed", C.c_uint64),
                ("max_iter", C.c_int32), ("max_outer", C.c_int32), ("inner_tol", C.c_double),
                ("check_every", C.c_int32), ("profile", C.c_int32), ("stream", C.c_void_p),
                ("precond", C.c_int32), ("precond_threshold", C.c_int32),
                ("factors", C.c_int32), ("apply_tc", C.c_int32), ("flexible", C.c_int32),
                ("schur_order", C.c_int32), ("krylov", C.c_int32), ("pad_", C.c_int32),
                ("auto_rho", C.c_double)]


class afn_build_info(C.Structure):
    _fields_ = [("n", C.c_int64), ("nr", C.c_int64), ("k", C.c_int64), ("d", C.c_int32),
                ("w", C.c_int32), ("kernel", C.c_int32), ("precision", C.c_int32),
                ("rank_r", C.c_int64), ("rank_branch", C.c_int32), ("precond", C.c_int32),
                ("l", C.c_double), ("mu", C.c_double), ("build_ms", C.c_double),
                ("device_bytes", C.c_int64), ("rho32", C.c_double)]


class afn_solve_info(C.Structure):
    _fields_ = [("iters", C.POINTER(C.c_int32)), ("relres", C.POINTER(C.c_double)),
                ("outer_steps", C.c_int32), ("converged", C.c_int32), ("solve_ms", C.c_double)]


class afn_system(C.Structure):
    _fields_ = [("points", C.c_void_p), ("n", C.c_int64), ("d", C.c_int32), ("kernel", C.c_int32),
                ("l", C.c_double), ("mu", C.c_double), ("k_max", C.c_int32),
                ("fsai_nnz", C.c_int32)]


class afn_batch_solve_info(C.Structure):
    _fields_ = [("converged", C.c_int32), ("columns", C.c_int32), ("graph_launches", C.c_int32),
                ("iters_max", C.c_int32), ("solve_ms", C.c_double), ("group_ms", C.c_double),
                ("single_ms", C.c_double), ("single_systems", C.c_int32), ("pad_", C.c_int32)]


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
        "afn_release_cached_memory": (None, []),
        "afn_set_wait_limit_ns": (None, [i64]),
        "afn_tune_set_cache": (i32, [C.c_char_p]),
        "afn_tune_get": (i32, [C.c_char_p, C.POINTER(i32)]),
        "afn_tune_put": (i32, [C.c_char_p, i32]),
        "afn_tune_count": (i32, []),
        "afn_tune_key": (i32, [i32, C.c_char_p, i32]),
        "afn_tune_clear": (None, []),
        "afn_kernel_matvec_noalloc": (i32, [P, i64, i32, i32, dbl, dbl, P, i32, P, P]),
        "afn_build_batched": (i32, [C.POINTER(afn_system), i32, C.POINTER(afn_options),
                                    C.POINTER(P)]),
        "afn_solve_batched": (i32, [P, P, C.POINTER(i32), dbl, P, P, P,
                                    C.POINTER(afn_batch_solve_info)]),
        "afn_batch_build_info": (i32, [P, i32, C.POINTER(afn_build_info)]),
        "afn_batch_build_ms": (dbl, [P]),
        "afn_batch_free": (None, [P]),
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
    """n x d row-major float64 points (a 2-D array)."""
    if _is_torch(a):
        import torch
        t = a.to(torch.float64).contiguous()
    else:
        t = np.ascontiguousarray(a, dtype=np.float64)
    if t.ndim != 2:
        raise ValueError("points must have shape (n, d), got %s" % (tuple(t.shape),))
    return t


def _f64_colmajor(a, n=None, what="block"):
    """n x m column-major float64 (as a contiguous m x n transpose buffer).  With
    ``n`` given, a block with another number of rows is refused: the library
    reads n x m values from the buffer and cannot see its size."""
    if not _is_torch(a):
        a = np.asarray(a, dtype=np.float64)
    nd = a.dim() if _is_torch(a) else a.ndim
    if nd not in (1, 2):
        raise ValueError("%s must have shape (n,) or (n, m)" % what)
    if n is not None and int(a.shape[0]) != int(n):
        raise ValueError("%s has %d rows, expected n = %d" % (what, int(a.shape[0]), int(n)))
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
    B, nrhs = _f64_colmajor(rhs, h.n, "rhs")
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
    """M^{-1} r (Alg. 3); r in PERMUTED order, (n,) or (n, nrhs).  FP64 handles
    apply in FP64, mixed handles run the FP32 apply of their solves."""
    R, nrhs = _f64_colmajor(r, h.n, "r")
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


def afn_release_cached_memory():
    """Return the library's cached device memory to the device (waits for idle)."""
    _lib.afn_release_cached_memory()


def afn_set_wait_limit_ns(ns: int):
    """Limit of the tensor-core kernels' bounded device waits (ns; <= 0 = 2 s)."""
    _lib.afn_set_wait_limit_ns(int(ns))


# --------------------------------------------------------------- autotuner --
def afn_tune_set_cache(path):
    """Persist the autotuner's choices in `path` (loaded if present); None stops."""
    _check(_lib.afn_tune_set_cache(None if path is None else str(path).encode()))


def afn_tune_get(key):
    v = C.c_int32(0)
    _check(_lib.afn_tune_get(key.encode(), C.byref(v)))
    return int(v.value)


def afn_tune_put(key, choice):
    _check(_lib.afn_tune_put(key.encode(), int(choice)))


def afn_tune_entries():
    """{key: choice} of every recorded decision."""
    out = {}
    buf = C.create_string_buffer(256)
    for i in range(_lib.afn_tune_count()):
        v = _lib.afn_tune_key(i, buf, 256)
        if v >= 0:
            out[buf.value.decode()] = int(v)
    return out


def afn_tune_clear():
    _lib.afn_tune_clear()


def afn_reset_kernel_stats(h: Handle):
    _check(_lib.afn_reset_kernel_stats(h.ptr))


# ------------------------------------------------------- operator entries --
def afn_kernel_matvec(points, kernel, l, mu, p, precision=PREC_FP64, stream=None):
    """(K + mu I) p, matrix-free; p (n,) or (n, nrhs)."""
    X = _f64_rowmajor(points)
    n, d = int(X.shape[0]), int(X.shape[1])
    Pm, nrhs = _f64_colmajor(p, n, "p")
    out = _empty_like_kind(Pm, tuple(Pm.shape), np.float64)
    px, kx = _ptr(X)
    pp, kp = _ptr(Pm)
    po, ko = _ptr(out)
    _check(_lib.afn_kernel_matvec(px, n, d, int(kernel), float(l), float(mu), pp, nrhs, po,
                                  int(precision), _stream_ptr(stream)))
    return out.T if out.ndim == 2 else out


def afn_kernel_matvec_noalloc(points, kernel, l, mu, p, q, stream=None):
    """FP64 (K + mu I) p into q without any device allocation (for callers
    whose device memory is planned up front, see include/afn.h).  points: a
    contiguous float64 CUDA tensor of shape (n, d).  p and q: contiguous
    float64 CUDA tensors of shape (nrhs, n) -- the storage of n x nrhs
    column-major blocks, one column per row of the tensor -- or of shape (n,)
    for one column.  Everything is checked before the library is called."""
    def need(ok, what):
        if not ok:
            raise ValueError("afn_kernel_matvec_noalloc: " + what)

    for name, t in (("points", points), ("p", p), ("q", q)):
        need(_is_torch(t), "%s must be a torch tensor" % name)
        need(str(t.dtype) == "torch.float64", "%s must be float64" % name)
        need(t.is_contiguous(), "%s must be contiguous" % name)
    need(points.dim() == 2, "points must have shape (n, d)")
    n, d = int(points.shape[0]), int(points.shape[1])
    need(p.dim() in (1, 2) and tuple(p.shape) == tuple(q.shape), "p and q must have one shape")
    if p.dim() == 1:
        need(int(p.shape[0]) == n, "p of shape (n,) must have n = %d entries" % n)
        nrhs = 1
    else:
        need(int(p.shape[1]) == n, "p and q must have shape (nrhs, n) with n = %d" % n)
        nrhs = int(p.shape[0])
    for name, t in (("points", points), ("p", p), ("q", q)):
        need(t.is_cuda, "%s must be in CUDA memory" % name)
    import torch
    cur = torch.cuda.current_device()
    for name, t in (("points", points), ("p", p), ("q", q)):
        need(t.device.index == cur, "%s must be on the current device (%d)" % (name, cur))
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


# ----------------------------------------------------------------- batches --
class Batch:
    """Owns an ``afn_batch*`` (many systems built together)."""

    def __init__(self, ptr, ns, ns_n):
        self.ptr = ptr
        self.nsys = ns
        self.n = ns_n

    def __del__(self):
        try:
            afn_batch_free(self)
        except Exception:
            pass


def afn_build_batched(systems, opt: afn_options | None = None, **kw):
    """Builds every system of ``systems`` (dicts with keys points, kernel, l,
    mu, k_max, fsai_nnz) with the options ``opt`` (precision AUTO unless
    given: MIXED or DF per system)."""
    if opt is None:
        kw.setdefault("precision", PREC_AUTO)
        opt = options(**kw)
    ns = len(systems)
    arr = (afn_system * ns)()
    keep = []
    for i, sy in enumerate(systems):
        X = _f64_rowmajor(sy["points"])
        px, kx = _ptr(X)
        keep.append(kx)
        arr[i] = afn_system(px, int(X.shape[0]), int(X.shape[1]), int(sy["kernel"]),
                            float(sy["l"]), float(sy["mu"]), int(sy["k_max"]), int(sy["fsai_nnz"]))
    b = C.c_void_p()
    _check(_lib.afn_build_batched(arr, ns, C.byref(opt), C.byref(b)))
    return Batch(b, ns, [int(sy["points"].shape[0]) for sy in systems])


def afn_batch_free(b: Batch):
    if b is not None and b.ptr:
        _lib.afn_batch_free(b.ptr)
        b.ptr = None


def afn_batch_build_info(b: Batch, system: int) -> afn_build_info:
    bi = afn_build_info()
    _check(_lib.afn_batch_build_info(b.ptr, int(system), C.byref(bi)))
    return bi


def afn_batch_build_ms(b: Batch) -> float:
    return float(_lib.afn_batch_build_ms(b.ptr))


def afn_solve_batched(b: Batch, rhs, tol):
    """Solves every system of the batch.  rhs: list of (n_s,) or (n_s, nrhs_s)
    arrays (all numpy, or all torch tensors on one device).  Returns (xs, info)
    with xs the list of solutions and info = dict(iters, relres (per system
    arrays), converged, columns, graph_launches, iters_max, solve_ms, status)."""
    if len(rhs) != b.nsys:
        raise ValueError("expected %d right-hand-side blocks" % b.nsys)
    cols = []
    nr = []
    for i, r in enumerate(rhs):
        Bc, m = _f64_colmajor(r, b.n[i], "rhs %d" % i)
        cols.append(Bc.reshape(-1))
        nr.append(m)
    if _is_torch(cols[0]):
        import torch
        flat = torch.cat(cols)
        out = torch.empty_like(flat)
    else:
        flat = np.concatenate(cols)
        out = np.empty_like(flat)
    tot = sum(nr)
    nrhs = (C.c_int32 * b.nsys)(*nr)
    its = np.zeros(tot, dtype=np.int32)
    rel = np.zeros(tot, dtype=np.float64)
    info = afn_batch_solve_info()
    pf, kf = _ptr(flat)
    po, ko = _ptr(out)
    st = _lib.afn_solve_batched(b.ptr, pf, nrhs, float(tol), po, _ptr(its)[0], _ptr(rel)[0],
                                C.byref(info))
    if st not in (AFN_OK, AFN_ERR_NO_CONVERGE):
        _check(st)
    xs, iters, relres = [], [], []
    o = c = 0
    for i in range(b.nsys):
        n, m = b.n[i], nr[i]
        blk = out[o:o + n * m].reshape(m, n)
        xs.append(blk.T if m > 1 or (_is_torch(rhs[i]) and rhs[i].dim() == 2) or
                  (not _is_torch(rhs[i]) and np.ndim(rhs[i]) == 2) else blk[0])
        iters.append(its[c:c + m].astype(np.int64))
        relres.append(rel[c:c + m].copy())
        o += n * m
        c += m
    return xs, dict(iters=iters, relres=relres, converged=info.converged, columns=info.columns,
                    graph_launches=info.graph_launches, iters_max=info.iters_max,
                    solve_ms=info.solve_ms, group_ms=info.group_ms, single_ms=info.single_ms,
                    single_systems=info.single_systems, status=st)


# ----------------------------------------------------------------- serving --
class afn_server_config(C.Structure):
    _fields_ = [("memory_budget", C.c_int64), ("max_active", C.c_int32),
                ("build_threads", C.c_int32), ("opt", afn_options)]


class afn_request_info(C.Structure):
    _fields_ = [("status", C.c_int32), ("converged", C.c_int32), ("nrhs", C.c_int32),
                ("pad_", C.c_int32), ("queue_ms", C.c_double), ("build_ms", C.c_double),
                ("wait_ms", C.c_double), ("solve_ms", C.c_double), ("latency_ms", C.c_double),
                ("device_bytes", C.c_int64)]


class afn_server_stats(C.Structure):
    _fields_ = [("submitted", C.c_int64), ("completed", C.c_int64), ("queued", C.c_int64),
                ("active", C.c_int32), ("peak_live", C.c_int32), ("graph_launches", C.c_int64),
                ("reserved_bytes", C.c_int64), ("peak_reserved_bytes", C.c_int64),
                ("budget_bytes", C.c_int64)]


def _bind_server():
    P, i64, i32, dbl = C.c_void_p, C.c_int64, C.c_int32, C.c_double
    sig = {
        "afn_server_default_config": (None, [C.POINTER(afn_server_config)]),
        "afn_server_create": (i32, [C.POINTER(afn_server_config), C.POINTER(P)]),
        "afn_server_submit": (i32, [P, C.POINTER(afn_system), P, i32, dbl, C.POINTER(i64)]),
        "afn_server_poll": (i32, [P, P, i32, C.POINTER(i32), i32]),
        "afn_server_result": (i32, [P, i64, P, P, P, C.POINTER(afn_request_info)]),
        "afn_server_get_stats": (i32, [P, C.POINTER(afn_server_stats)]),
        "afn_server_destroy": (None, [P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(_lib, name)
        f.restype = res
        f.argtypes = args


_bind_server()


class Server:
    """A serving loop (``afn_server*``): submit systems at any time, poll for
    finished ones, fetch results.  Options are those of ``options`` (mixed
    precision); memory_budget (bytes, 0 = half the free device memory),
    max_active and build_threads as in afn_server_config."""

    def __init__(self, memory_budget=0, max_active=0, build_threads=8, **kw):
        cfg = afn_server_config()
        _lib.afn_server_default_config(C.byref(cfg))
        cfg.memory_budget = int(memory_budget)
        cfg.max_active = int(max_active)
        cfg.build_threads = int(build_threads)
        kw.setdefault("precision", PREC_AUTO)
        cfg.opt = options(**kw)
        self.ptr = C.c_void_p()
        _check(_lib.afn_server_create(C.byref(cfg), C.byref(self.ptr)))
        self._shape = {}

    def submit(self, system, rhs, tol):
        """system: dict(points, kernel, l, mu, k_max, fsai_nnz); rhs (n,) or
        (n, nrhs).  Returns the request id."""
        X = _f64_rowmajor(system["points"])
        Bc, m = _f64_colmajor(rhs, X.shape[0], "rhs")
        px, kx = _ptr(X)
        pb, kb = _ptr(Bc)
        sy = afn_system(px, int(X.shape[0]), int(X.shape[1]), int(system["kernel"]),
                        float(system["l"]), float(system["mu"]), int(system["k_max"]),
                        int(system["fsai_nnz"]))
        rid = C.c_int64(0)
        _check(_lib.afn_server_submit(self.ptr, C.byref(sy), pb, m, float(tol), C.byref(rid)))
        self._shape[int(rid.value)] = (int(X.shape[0]), m, np.ndim(rhs) if not _is_torch(rhs)
                                       else rhs.dim())
        return int(rid.value)

    def poll(self, max_ids=1024, wait_ms=0):
        """Ids of requests finished since the last poll."""
        ids = np.zeros(max(1, int(max_ids)), dtype=np.int64)
        cnt = C.c_int32(0)
        _check(_lib.afn_server_poll(self.ptr, _ptr(ids)[0], int(max_ids), C.byref(cnt),
                                    int(wait_ms)))
        return [int(v) for v in ids[: cnt.value]]

    def result(self, rid):
        """(x, info) of a finished request; x (n,) or (n, nrhs) float64 host."""
        n, m, nd = self._shape.pop(int(rid))
        x = np.zeros((m, n), dtype=np.float64)
        its = np.zeros(m, dtype=np.int32)
        rel = np.zeros(m, dtype=np.float64)
        inf = afn_request_info()
        st = _lib.afn_server_result(self.ptr, int(rid), _ptr(x)[0], _ptr(its)[0], _ptr(rel)[0],
                                    C.byref(inf))
        if st not in (AFN_OK, AFN_ERR_NO_CONVERGE):
            _check(st)
        info = {f: getattr(inf, f) for f, _ in afn_request_info._fields_ if f != "pad_"}
        info.update(iters=its.astype(np.int64), relres=rel, status=st)
        return (x.T if nd == 2 else x[0]), info

    def stats(self):
        s = afn_server_stats()
        _check(_lib.afn_server_get_stats(self.ptr, C.byref(s)))
        return {f: getattr(s, f) for f, _ in afn_server_stats._fields_}

    def close(self):
        if self.ptr:
            _lib.afn_server_destroy(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
