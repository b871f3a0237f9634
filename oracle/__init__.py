"""Plain FP64 CPU oracle for AFN-preconditioned CG (arXiv 2304.05460).

TEST INFRASTRUCTURE ONLY.  Only the test-suite, ``__graft_entry__.smoke()``
and the benchmark's CPU-baseline / reference arm may import this package.
The CUDA library never imports, links or loads it, and it never imports the
CUDA library; the two share nothing but the seeded input generators.

The arithmetic lives in ``afn_oracle.c`` (one C file, FP64, no BLAS,
``-ffp-contract=off``); this module compiles it with gcc on first use and
marshals numpy arrays through ctypes.  Each wrapper names the passage of the
paper its C function restates.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "afn_oracle.c")
_SO = os.path.join(_HERE, "libafn_oracle.so")
_lock = threading.Lock()
_lib = None

GAUSSIAN = 0
MATERN32 = 1

OK, ERR_ARG, ERR_NOT_SPD, ERR_NO_CONVERGE = 0, 1, 3, 4


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/libafn_oracle.so`` (gcc, OpenMP)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + ".tmp.%d" % os.getpid()
        cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
               "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _SO)
    return _SO


def _L():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = C.CDLL(_SO)
            P = C.c_void_p
            i64, i32, dbl, u64 = C.c_int64, C.c_int, C.c_double, C.c_uint64
            sig = {
                "orc_set_threads": (None, [i32]),
                "orc_get_threads": (i32, []),
                "orc_sqdist": (dbl, [P, P, i32]),
                "orc_kernel_from_sqdist": (dbl, [dbl, i32, dbl]),
                "orc_kernel_eval": (dbl, [P, P, i32, i32, dbl]),
                "orc_kernel_matrix": (None, [P, i64, P, i64, i32, i32, dbl, P]),
                "orc_matvec": (None, [P, i64, i32, i32, dbl, dbl, P, i32, P]),
                "orc_jacobi_eig": (None, [P, i64, P, P]),
                "orc_nystrom_build": (i32, [P, i64, i32, i32, dbl, i64, P, P, P]),
                "orc_nystrom_apply": (None, [i64, i64, i64, P, P, dbl, P, P]),
                "orc_pcg_nystrom": (i32, [P, i64, i32, i32, dbl, dbl, i64, i64, P, P, P, dbl, i32,
                                          i32, P, P, P]),
                "orc_fps": (i32, [P, i64, i32, i64, i64, P]),
                "orc_fps_centroid_start": (i64, [P, i64, i32]),
                "orc_splitmix64_next": (u64, [P]),
                "orc_uniform_sample": (i32, [i64, i64, u64, P]),
                "orc_permutation": (i32, [i64, P, i64, P]),
                "orc_knn_pattern": (None, [P, i64, i32, i32, P, P]),
                "orc_cholesky": (i32, [P, i64, P]),
                "orc_forward": (None, [P, i64, P, P]),
                "orc_backward": (None, [P, i64, P, P]),
                "orc_fsai_row": (i32, [P, i32, P]),
                "orc_afn_build": (i32, [P, i64, i32, i32, dbl, dbl, i64, i32, P, P, P, P, P, P, P]),
                "orc_afn_apply": (None, [i64, i64, i32, P, P, P, P, P, P]),
                "orc_dense_M_factored": (None, [i64, i64, i32, P, P, P, P, P]),
                "orc_dense_M_expanded": (None, [P, i64, i32, i32, dbl, dbl, i64, i32, P, P, P, P, P]),
                "orc_pcg": (i32, [P, i64, i32, i32, dbl, dbl, i64, i32, P, P, P, P, P, dbl, i32, i32,
                                  P, P, P]),
                "orc_dense_solve": (i32, [P, i64, i32, i32, dbl, dbl, P, i32, P]),
                "orc_tridiagonalize": (None, [P, i64, P, P]),
                "orc_sturm_count": (i64, [P, P, i64, dbl]),
                "orc_tridiag_max_eig": (dbl, [P, P, i64]),
                "orc_rank_estimate": (i64, [P, i64, i32, i32, dbl, dbl, i64, u64, i64, P, P]),
            }
            for name, (res, args) in sig.items():
                f = getattr(lib, name)
                f.restype = res
                f.argtypes = args
            _lib = lib
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _kid(kernel):
    if isinstance(kernel, str):
        return {"gaussian": GAUSSIAN, "matern32": MATERN32}[kernel]
    return int(kernel)


def set_threads(t: int) -> None:
    _L().orc_set_threads(int(t))


def get_threads() -> int:
    return int(_L().orc_get_threads())


# --------------------------------------------------------------------------
# kernels (eq. (gaussianf); Sec. 5 kernel list)
# --------------------------------------------------------------------------
def kernel_from_sqdist(r2: float, kernel, l: float) -> float:
    return float(_L().orc_kernel_from_sqdist(float(r2), _kid(kernel), float(l)))


def kernel_matrix(X, Y, kernel, l):
    X, Y = _f64(X), _f64(Y)
    out = np.empty((X.shape[0], Y.shape[0]), dtype=np.float64)
    _L().orc_kernel_matrix(_p(X), X.shape[0], _p(Y), Y.shape[0], X.shape[1], _kid(kernel),
                           float(l), _p(out))
    return out


def matvec(X, kernel, l, mu, p):
    """(K + mu I) p, matrix-free; p is (n,) or (n, nrhs)."""
    X = _f64(X)
    p = np.asarray(p, dtype=np.float64)
    one = p.ndim == 1
    P = np.asfortranarray(p.reshape(p.shape[0], -1))
    out = np.empty_like(P, order="F")
    _L().orc_matvec(_p(X), X.shape[0], X.shape[1], _kid(kernel), float(l), float(mu),
                    _p(P), P.shape[1], _p(out))
    return out[:, 0].copy() if one else np.ascontiguousarray(out)


# --------------------------------------------------------------------------
# landmarks (Alg. 6, uniform sampling of Alg. 2) and the permutation (Sec. 2)
# --------------------------------------------------------------------------
def fps(X, k, start=0):
    X = _f64(X)
    idx = np.empty(max(int(k), 1), dtype=np.int64)
    st = _L().orc_fps(_p(X), X.shape[0], X.shape[1], int(k), int(start), _p(idx))
    if st:
        raise ValueError("oracle fps: bad arguments")
    return idx[: int(k)].copy()


def fps_centroid_start(X):
    X = _f64(X)
    return int(_L().orc_fps_centroid_start(_p(X), X.shape[0], X.shape[1]))


def splitmix64_stream(seed, count):
    st = np.array([seed], dtype=np.uint64)
    return np.array([_L().orc_splitmix64_next(_p(st)) for _ in range(count)], dtype=np.uint64)


def uniform_sample(n, k, seed):
    idx = np.empty(max(int(k), 1), dtype=np.int64)
    if _L().orc_uniform_sample(int(n), int(k), C.c_uint64(int(seed) & (2**64 - 1)), _p(idx)):
        raise ValueError("oracle uniform_sample: bad arguments")
    return idx[: int(k)].copy()


def permutation(n, landmarks):
    lm = np.ascontiguousarray(landmarks, dtype=np.int64)
    perm = np.empty(int(n), dtype=np.int64)
    if _L().orc_permutation(int(n), _p(lm), lm.shape[0], _p(perm)):
        raise ValueError("oracle permutation: bad landmarks")
    return perm


def knn_pattern(Xr, w):
    Xr = _f64(Xr)
    nr = Xr.shape[0]
    pat = np.empty((max(nr, 1), w), dtype=np.int32)
    rl = np.empty(max(nr, 1), dtype=np.int32)
    _L().orc_knn_pattern(_p(Xr), nr, Xr.shape[1], int(w), _p(pat), _p(rl))
    return pat[:nr].copy(), rl[:nr].copy()


# --------------------------------------------------------------------------
# dense factorisations (Alg. 2 Cholesky; Alg. 1 FSAI row)
# --------------------------------------------------------------------------
def cholesky(A):
    A = _f64(A)
    k = A.shape[0]
    Lo = np.empty_like(A)
    st = _L().orc_cholesky(_p(A), k, _p(Lo))
    if st:
        raise np.linalg.LinAlgError("oracle cholesky: not SPD")
    return Lo


def forward(Lo, b):
    Lo, b = _f64(Lo), _f64(b)
    x = np.empty_like(b)
    _L().orc_forward(_p(Lo), Lo.shape[0], _p(b), _p(x))
    return x


def backward(Lo, b):
    Lo, b = _f64(Lo), _f64(b)
    x = np.empty_like(b)
    _L().orc_backward(_p(Lo), Lo.shape[0], _p(b), _p(x))
    return x


def fsai_row(A):
    A = _f64(A)
    g = np.empty(A.shape[0], dtype=np.float64)
    if _L().orc_fsai_row(_p(A), A.shape[0], _p(g)):
        raise np.linalg.LinAlgError("oracle fsai_row: pattern block not SPD")
    return g


# --------------------------------------------------------------------------
# AFN (Alg. 2 build, Alg. 3 apply, eq. (factorized-form) and eq. (realM))
# --------------------------------------------------------------------------
def landmarks_for(X, k, mode="fps", start=0, seed=0):
    """Landmark indices: FPS (Alg. 6, start index or 'centroid') or uniform."""
    n = X.shape[0]
    if k == 0:
        return np.empty(0, dtype=np.int64)
    if mode == "fps":
        s = fps_centroid_start(X) if start == "centroid" else int(start)
        return fps(X, k, s)
    if mode == "uniform":
        return uniform_sample(n, k, seed)
    raise ValueError(mode)


def afn_build(X, kernel, l, mu, k, w, landmarks=None, mode="fps", start=0, seed=0):
    """Alg. 2.  Returns a dict with perm, Xp (permuted points), L, K12,
    pattern, rowlen, G, k, nr, w.  Raises LinAlgError if a block is not SPD."""
    X = _f64(X)
    n, d = X.shape
    k = int(min(max(k, 0), n))
    nr = n - k
    w = int(max(1, min(w, max(nr, 1))))
    lm = landmarks_for(X, k, mode, start, seed) if landmarks is None else np.asarray(landmarks, np.int64)
    lm = np.ascontiguousarray(lm, dtype=np.int64)
    perm = np.empty(n, dtype=np.int64)
    Lo = np.zeros((max(k, 1), max(k, 1)))
    K12 = np.zeros((max(k, 1), max(nr, 1)))
    pat = np.full((max(nr, 1), w), -1, dtype=np.int32)
    rl = np.zeros(max(nr, 1), dtype=np.int32)
    G = np.zeros((max(nr, 1), w))
    st = _L().orc_afn_build(_p(X), n, d, _kid(kernel), float(l), float(mu), k, w, _p(lm),
                            _p(perm), _p(Lo), _p(K12), _p(pat), _p(rl), _p(G))
    if st == ERR_ARG:
        raise ValueError("oracle afn_build: bad arguments")
    if st == ERR_NOT_SPD:
        raise np.linalg.LinAlgError("oracle afn_build: not SPD")
    return dict(perm=perm, Xp=X[perm], L=Lo[:k, :k].copy(), K12=K12[:k, :nr].copy(),
                pattern=pat[:nr].copy(), rowlen=rl[:nr].copy(), G=G[:nr].copy(),
                k=k, nr=nr, w=w, landmarks=lm.copy(), kernel=_kid(kernel), l=float(l),
                mu=float(mu))


def _fac_args(f):
    k, nr, w = f["k"], f["nr"], f["w"]
    Lo = _f64(f["L"]) if k > 0 else np.zeros((1, 1))
    K12 = _f64(f["K12"]) if k > 0 and nr > 0 else np.zeros((1, 1))
    pat = np.ascontiguousarray(f["pattern"], dtype=np.int32) if nr > 0 else np.full((1, w), -1, np.int32)
    G = _f64(f["G"]) if nr > 0 else np.zeros((1, w))
    return k, nr, w, Lo, K12, pat, G


def afn_apply(f, r):
    """Alg. 3: s = M^{-1} r, vectors in the permuted order."""
    k, nr, w, Lo, K12, pat, G = _fac_args(f)
    r = _f64(r)
    s = np.empty_like(r)
    _L().orc_afn_apply(k, nr, w, _p(Lo), _p(K12), _p(pat), _p(G), _p(r), _p(s))
    return s


def dense_M_factored(f):
    k, nr, w, Lo, K12, pat, G = _fac_args(f)
    n = k + nr
    M = np.empty((n, n))
    _L().orc_dense_M_factored(k, nr, w, _p(Lo), _p(K12), _p(pat), _p(G), _p(M))
    return M


def dense_M_expanded(f):
    k, nr, w, Lo, K12, pat, G = _fac_args(f)
    Xp = _f64(f["Xp"])
    n, d = Xp.shape
    M = np.empty((n, n))
    _L().orc_dense_M_expanded(_p(Xp), n, d, f["kernel"], f["l"], f["mu"], k, w, _p(Lo), _p(K12),
                              _p(pat), _p(G), _p(M))
    return M


def pcg(f, b, tol, max_iter=500, max_restarts=3, identity=False):
    """PCG with the AFN preconditioner of ``f`` (or none when identity=True)
    on (K + mu I) x = b, b in ORIGINAL point order, one or more columns.
    Returns (x, iters, relres, status) with per-column arrays."""
    k, nr, w, Lo, K12, pat, G = _fac_args(f)
    Xp = _f64(f["Xp"])
    n, d = Xp.shape
    perm = f["perm"]
    b = np.asarray(b, dtype=np.float64)
    one = b.ndim == 1
    B = b.reshape(n, -1)
    X = np.zeros_like(B)
    its = np.zeros(B.shape[1], dtype=np.int64)
    rel = np.zeros(B.shape[1])
    sts = np.zeros(B.shape[1], dtype=np.int64)
    for c in range(B.shape[1]):
        bp = np.ascontiguousarray(B[perm, c])
        xp = np.empty(n)
        it = C.c_int(0)
        rr = C.c_double(0.0)
        nulls = (None, None, None, None) if identity else (_p(Lo), _p(K12), _p(pat), _p(G))
        st = _L().orc_pcg(_p(Xp), n, d, f["kernel"], f["l"], f["mu"], 0 if identity else k, w,
                          *nulls, _p(bp), float(tol), int(max_iter), int(max_restarts), _p(xp),
                          C.byref(it), C.byref(rr))
        X[perm, c] = xp
        its[c], rel[c], sts[c] = it.value, rr.value, st
    if one:
        return X[:, 0], int(its[0]), float(rel[0]), int(sts[0])
    return X, its, rel, sts


def jacobi_eig(A):
    """Cyclic Jacobi (Golub & Van Loan Alg. 8.5.3): eigenvalues w and
    eigenvectors V (columns) of the symmetric matrix A."""
    A = np.array(A, dtype=np.float64, order="C")
    m = A.shape[0]
    V = np.empty((m, m))
    w = np.empty(m)
    _L().orc_jacobi_eig(_p(A), m, _p(V), _p(w))
    return w, V


def nystrom_build(X, kernel, l, mu, k, landmarks=None, mode="fps", start=0, seed=0):
    """Column-sampling Nystrom preconditioner (Sec. 2) in the orthonormal form
    of eq. (nystrom1-smw): U (n x r, permuted order, landmarks first) and
    Lambda (r) with U Lambda U^T = K_nys.  Raises LinAlgError if K_SS is not SPD."""
    X = _f64(X)
    n, d = X.shape
    k = int(min(max(k, 0), n))
    lm = landmarks_for(X, k, mode, start, seed) if landmarks is None else np.asarray(landmarks, np.int64)
    lm = np.ascontiguousarray(lm, dtype=np.int64)
    perm = np.empty(n, dtype=np.int64)
    _L().orc_permutation(n, _p(lm), k, _p(perm))
    Xp = np.ascontiguousarray(X[perm])
    U = np.zeros((n, max(k, 1)))
    lam = np.zeros(max(k, 1))
    r = C.c_int64(0)
    st = _L().orc_nystrom_build(_p(Xp), n, d, _kid(kernel), float(l), k, _p(U), _p(lam),
                                C.byref(r))
    if st == ERR_NOT_SPD:
        raise np.linalg.LinAlgError("oracle nystrom_build: K_SS + nu I not SPD")
    r = int(r.value)
    return dict(precond="nystrom", perm=perm, Xp=Xp, U=U[:, :max(k, 1)], lam=lam, k=k, r=r,
                landmarks=lm.copy(), kernel=_kid(kernel), l=float(l), mu=float(mu))


def nystrom_apply(f, rv):
    """eq. (nystrom1-smw): s = U (Lambda + mu I)^{-1} U^T r + (r - U U^T r) / mu, permuted order."""
    rv = _f64(rv)
    s = np.empty_like(rv)
    n = f["Xp"].shape[0]
    _L().orc_nystrom_apply(n, max(f["k"], 1), f["r"], _p(_f64(f["U"])), _p(_f64(f["lam"])),
                           float(f["mu"]), _p(rv), _p(s))
    return s


def pcg_nystrom(f, b, tol, max_iter=500, max_restarts=3):
    """PCG with the Nystrom preconditioner of ``f`` (Alg. 5, k < 2000 branch),
    b in ORIGINAL point order; returns (x, iters, relres, status) per column."""
    Xp = _f64(f["Xp"])
    n, d = Xp.shape
    perm = f["perm"]
    b = np.asarray(b, dtype=np.float64)
    one = b.ndim == 1
    B = b.reshape(n, -1)
    X = np.zeros_like(B)
    its = np.zeros(B.shape[1], dtype=np.int64)
    rel = np.zeros(B.shape[1])
    sts = np.zeros(B.shape[1], dtype=np.int64)
    for c in range(B.shape[1]):
        bp = np.ascontiguousarray(B[perm, c])
        xp = np.empty(n)
        it = C.c_int(0)
        rr = C.c_double(0.0)
        st = _L().orc_pcg_nystrom(_p(Xp), n, d, f["kernel"], f["l"], f["mu"], max(f["k"], 1),
                                  f["r"], _p(_f64(f["U"])), _p(_f64(f["lam"])), _p(bp),
                                  float(tol), int(max_iter), int(max_restarts), _p(xp),
                                  C.byref(it), C.byref(rr))
        X[perm, c] = xp
        its[c], rel[c], sts[c] = it.value, rr.value, st
    if one:
        return X[:, 0], int(its[0]), float(rel[0]), int(sts[0])
    return X, its, rel, sts


def strategy(X, kernel, l, mu, k_max, w, m=1000, seed=0, threshold=2000):
    """Alg. 5: estimate k by Alg. 4; k < threshold (2000 in the paper): the
    Nystrom preconditioner with k landmarks, else AFN.  Returns the factors
    (``precond`` = "nystrom" or "afn")."""
    k = rank_estimate(X, kernel, l, mu, m=m, seed=seed, k_max=k_max)[0]
    if k < threshold:
        return nystrom_build(X, kernel, l, mu, k)
    f = afn_build(X, kernel, l, mu, k, w)
    f["precond"] = "afn"
    return f


def dense_solve(X, kernel, l, mu, b):
    """a* = (K + mu I)^{-1} b by a dense Cholesky factorisation (eq. (Problem))."""
    X = _f64(X)
    b = np.asarray(b, dtype=np.float64)
    one = b.ndim == 1
    B = np.asfortranarray(b.reshape(X.shape[0], -1))
    out = np.empty_like(B, order="F")
    st = _L().orc_dense_solve(_p(X), X.shape[0], X.shape[1], _kid(kernel), float(l), float(mu),
                              _p(B), B.shape[1], _p(out))
    if st:
        raise np.linalg.LinAlgError("oracle dense_solve: not SPD")
    return out[:, 0].copy() if one else np.ascontiguousarray(out)


def true_relres(X, kernel, l, mu, x, b):
    """||b - (K + mu I) x||_2 / ||b||_2 per column, in FP64 (the relative
    residual of the stopping test, Sec. 5).  A zero column b has the solution
    x = 0: its value is 0 when the residual is zero and +inf otherwise."""
    x = np.asarray(x, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    r = b.reshape(b.shape[0], -1) - matvec(X, kernel, l, mu, x.reshape(x.shape[0], -1)).reshape(b.shape[0], -1)
    nr = np.linalg.norm(r, axis=0)
    nb = np.linalg.norm(b.reshape(b.shape[0], -1), axis=0)
    out = np.where(nr == 0.0, 0.0, np.inf)
    np.divide(nr, nb, out=out, where=nb > 0)
    return out


# --------------------------------------------------------------------------
# eigenvalue tools and Alg. 4
# --------------------------------------------------------------------------
def tridiagonalize(A):
    A = np.array(A, dtype=np.float64, copy=True, order="C")
    m = A.shape[0]
    dg = np.empty(max(m, 1))
    of = np.zeros(max(m - 1, 1))
    _L().orc_tridiagonalize(_p(A), m, _p(dg), _p(of))
    return dg[:m].copy(), of[: max(m - 1, 0)].copy()


def sturm_count(dg, of, sigma):
    dg, of = _f64(dg), _f64(of if len(of) else np.zeros(1))
    return int(_L().orc_sturm_count(_p(dg), _p(of), dg.shape[0], float(sigma)))


def tridiag_max_eig(dg, of):
    dg, of = _f64(dg), _f64(of if len(of) else np.zeros(1))
    return float(_L().orc_tridiag_max_eig(_p(dg), _p(of), dg.shape[0]))


def rank_estimate(X, kernel, l, mu, m=1000, seed=0, k_max=4000):
    """Alg. 4 (readings in the C source).  Returns (k, r, branch)."""
    X = _f64(X)
    r = C.c_int64(0)
    br = C.c_int(0)
    k = _L().orc_rank_estimate(_p(X), X.shape[0], X.shape[1], _kid(kernel), float(l), float(mu),
                               int(m), C.c_uint64(int(seed) & (2**64 - 1)), int(k_max),
                               C.byref(r), C.byref(br))
    return int(k), int(r.value), int(br.value)


# --------------------------------------------------------------------------
# sampled outputs (large problems)
# --------------------------------------------------------------------------
def _sig_sampled(lib):
    P, i64, i32, dbl = C.c_void_p, C.c_int64, C.c_int, C.c_double
    lib.orc_matvec_rows.restype = None
    lib.orc_matvec_rows.argtypes = [P, i64, i32, i32, dbl, dbl, P, i32, P, i64, P]
    lib.orc_fsai_rows.restype = i32
    lib.orc_fsai_rows.argtypes = [P, i64, i32, i32, dbl, dbl, i64, i32, P, P, P, i64, P]
    lib.orc_knn_rows.restype = None
    lib.orc_knn_rows.argtypes = [P, i64, i32, i32, P, i64, P]


def matvec_rows(X, kernel, l, mu, p, rows):
    """Rows `rows` of (K + mu I) p (p: (n,) or (n, nrhs)); returns (len(rows), nrhs)."""
    lib = _L()
    _sig_sampled(lib)
    X = _f64(X)
    P = np.asfortranarray(np.asarray(p, dtype=np.float64).reshape(X.shape[0], -1))
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    if rows.size and (rows.min() < 0 or rows.max() >= X.shape[0]):
        raise ValueError("matvec_rows: row index out of range")
    out = np.empty((rows.shape[0], P.shape[1]), order="F")
    lib.orc_matvec_rows(_p(X), X.shape[0], X.shape[1], _kid(kernel), float(l), float(mu), _p(P),
                        P.shape[1], _p(rows), rows.shape[0], _p(out))
    return np.ascontiguousarray(out)


def knn_rows(Xr, w, rows):
    """Rows `rows` of the FSAI pattern of Xr (Sec. 3.1), (len(rows), w) int32."""
    lib = _L()
    _sig_sampled(lib)
    Xr = _f64(Xr)
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    if rows.size and (rows.min() < 0 or rows.max() >= Xr.shape[0]):
        raise ValueError("knn_rows: row index out of range")
    out = np.empty((max(rows.shape[0], 1), int(w)), dtype=np.int32)
    lib.orc_knn_rows(_p(Xr), Xr.shape[0], Xr.shape[1], int(w), _p(rows), rows.shape[0], _p(out))
    return out[: rows.shape[0]].copy()


def fsai_rows(Xp, kernel, l, mu, k, w, Lo, pattern, rows):
    """FSAI rows (Alg. 1 on the Schur complement) for the given Schur rows."""
    lib = _L()
    _sig_sampled(lib)
    Xp = _f64(Xp)
    Lo = _f64(Lo) if k > 0 else np.zeros((1, 1))
    pat = np.ascontiguousarray(pattern, dtype=np.int32)
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    out = np.zeros((rows.shape[0], w))
    st = lib.orc_fsai_rows(_p(Xp), Xp.shape[0], Xp.shape[1], _kid(kernel), float(l), float(mu),
                           int(k), int(w), _p(Lo), _p(pat), _p(rows), rows.shape[0], _p(out))
    if st == 1:
        raise ValueError("oracle fsai_rows: k, w or a row index out of range")
    if st:
        raise np.linalg.LinAlgError("oracle fsai_rows: not SPD")
    return out
