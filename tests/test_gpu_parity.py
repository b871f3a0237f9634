"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Bars:
  * FPS indices, permutation and FSAI pattern: bit-exact.
  * FP64 path L, W and G: max |gpu - oracle| <= 1e-10 max |oracle|; the same
    bar for G of mixed handles built with FP64 factors.
  * Solves: the final relative residual ||b - (K + mu I) x|| / ||b||,
    recomputed by the oracle in FP64, is <= tol; FP64 iteration counts are
    within +-2 of the oracle's.
  * FP64 matvec: |gpu - oracle| <= 1e-12 (sum_j |K_ij p_j| + mu |p_i|) per
    entry; FP32 matvec: <= 2e-5 of the same scale (the FP32 evaluation of
    r^2, 2^x and the accumulation, each a few ulp of 2^-24 amplified by d
    and the summation length).
"""
import numpy as np
import pytest

import oracle
from paper_2304_05460_gb300 import inputs

pytestmark = pytest.mark.gpu

G, M32 = 0, 1


@pytest.fixture(scope="module")
def afn():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2304_05460_gb300 import afn as a
    return a


def scale_bound(X, ker, l, mu, p):
    """sum_j |K_ij p_j| + mu |p_i| (FP64, oracle kernel values)."""
    K = oracle.kernel_matrix(X, X, ker, l)
    P = np.abs(np.asarray(p).reshape(X.shape[0], -1))
    return K @ P + mu * P


# ------------------------------------------------------------------ FPS ---
@pytest.mark.parametrize("n,d,k,start", [(1, 3, 1, 0), (37, 1, 37, 5), (1000, 3, 200, 0),
                                         (3001, 5, 257, 17), (2500, 16, 300, 0),
                                         (4097, 8, 1000, 0)])
def test_fps_bit_exact(afn, n, d, k, start):
    X = inputs.normal_points(n, d, 100 + n)
    assert np.array_equal(afn.afn_fps(X, k, start), oracle.fps(X, k, start))


def test_fps_ties_duplicates_centroid(afn):
    g = np.stack(np.meshgrid(np.arange(6.0), np.arange(6.0), indexing="ij"), -1).reshape(-1, 2)
    X = np.concatenate([g, g[:10]])          # exact ties and duplicated points
    assert np.array_equal(afn.afn_fps(X, len(X), 0), oracle.fps(X, len(X), 0))
    Y = inputs.uniform_points(777, 3, 5)
    c = oracle.fps_centroid_start(Y)
    assert np.array_equal(afn.afn_fps(Y, 50, -1), oracle.fps(Y, 50, c))


def test_fps_full_size_normal_8d(afn):
    s = inputs.normal_8d(l=1.0, nrhs=1)
    assert np.array_equal(afn.afn_fps(s.X, 4000, 0), oracle.fps(s.X, 4000, 0))


# ------------------------------------------------------------------ KNN ---
@pytest.mark.parametrize("nr,d,w", [(1, 3, 1), (50, 2, 1), (300, 3, 32), (1500, 8, 64),
                                    (700, 16, 50), (129, 3, 200)])
def test_knn_bit_exact(afn, nr, d, w):
    X = inputs.uniform_points(nr, d, 200 + nr)
    pat, _ = oracle.knn_pattern(X, w)
    assert np.array_equal(afn.afn_knn_pattern(X, w), pat)


def test_knn_ties_lattice(afn):
    g = np.stack(np.meshgrid(np.arange(7.0), np.arange(7.0), indexing="ij"), -1).reshape(-1, 2)
    X = g[inputs.rng(3).permutation(len(g))]
    pat, _ = oracle.knn_pattern(X, 9)
    assert np.array_equal(afn.afn_knn_pattern(X, 9), pat)


def _pattern_layout_ok(pat, w):
    """Row i: min(i, w-1) neighbours j < i, then i itself, then -1 padding."""
    nr = pat.shape[0]
    i = np.arange(nr)
    m = np.minimum(i, w - 1)
    assert np.array_equal(pat[i, m], i)
    pad = np.arange(w)[None, :] > m[:, None]
    assert np.all(pat[pad] == -1)
    used = (np.arange(w)[None, :] < m[:, None])
    assert np.all((pat[used] >= 0) & (pat[used] < np.repeat(i, w).reshape(nr, w)[used]))


def _sample_rows(nr, w, seed, count):
    g = inputs.rng(seed)
    edge = [0, 1, w - 2, w - 1, w, nr // 2, nr - 3, nr - 2, nr - 1]
    return np.unique(np.concatenate([[r for r in edge if 0 <= r < nr],
                                     g.choice(nr, size=min(count, nr), replace=False)]))


def test_knn_prefix_full_size(afn):
    # row i depends only on points 0..i: the oracle checks a prefix exactly, and
    # sampled rows over the whole range (the last rows included) one by one
    X = inputs.clusters_3d(nrhs=1).X
    full = afn.afn_knn_pattern(X, 50)
    pat, _ = oracle.knn_pattern(X[:6000], 50)
    assert np.array_equal(full[:6000], pat)
    _pattern_layout_ok(full, 50)
    rows = _sample_rows(len(X), 50, 31, 300)
    assert np.array_equal(full[rows], oracle.knn_rows(X, 50, rows))


@pytest.mark.parametrize("which", ["normal_8d", "clusters_3d"])
def test_knn_pattern_of_full_size_builds(afn, which):
    # the FSAI pattern of the handles the benchmark builds: n = 50k (Alg. 4 k = 4000 at
    # l = 1, n_r = 46,000, w = 64) and n = 200k (k = 2000, n_r = 198,000, w = 50), in the
    # handle's Schur-row order; sampled rows over the whole range against the oracle
    if which == "normal_8d":
        s = inputs.normal_8d(l=1.0, nrhs=1)
        h = afn.afn_build(s.X, G, 1.0, 1e-2, 4000, 64, precision=afn.PREC_MIXED,
                          rank_mode=afn.RANK_ESTIMATE, rank_subsample=1000, seed=s.seed)
    else:
        s = inputs.clusters_3d(nrhs=1)
        h = afn.afn_build(s.X, s.kernel, s.l, s.mu, s.k, s.w, precision=afn.PREC_MIXED)
    bi = h.info
    perm = afn.afn_get_perm(h)
    pat, _ = afn.afn_get_G(h)
    Xr = s.X[perm[bi.k:]]
    _pattern_layout_ok(pat, bi.w)
    rows = _sample_rows(bi.nr, bi.w, 37, 250)
    assert np.array_equal(pat[rows], oracle.knn_rows(Xr, bi.w, rows))
    assert np.array_equal(afn.afn_knn_pattern(Xr, bi.w), pat)
    afn.afn_free(h)


# --------------------------------------------------------------- matvec ---
@pytest.mark.parametrize("n,d,ker,nrhs", [(1, 3, G, 1), (257, 3, G, 1), (1000, 8, M32, 3),
                                          (2049, 16, G, 5), (1500, 2, M32, 33)])
def test_matvec_fp64(afn, n, d, ker, nrhs):
    X = inputs.normal_points(n, d, 300 + n)
    P = inputs.rhs(n, nrhs, 301 + n)
    l = 0.7 * np.sqrt(d)
    ref = oracle.matvec(X, ker, l, 1e-2, P)
    # FP64 kernel, and the double-float kernel (FP32 pipes) of the mixed
    # solves' residual replacements: both within 1e-12 of the scale
    for prec in (afn.PREC_FP64, afn.MATVEC_DF):
        q = afn.afn_kernel_matvec(X, ker, l, 1e-2, P, precision=prec)
        bound = scale_bound(X, ker, l, 1e-2, P).reshape(q.shape)
        err = np.abs(q - ref.reshape(q.shape)) / (bound + 1e-300)
        assert err.max() <= 1e-12, (prec, err.max())


@pytest.mark.parametrize("n,d,ker,nrhs", [(1, 3, G, 8), (31, 3, M32, 9), (2049, 16, G, 8),
                                          (777, 8, M32, 40), (1000, 3, G, 32), (1500, 2, M32, 64),
                                          (4097, 8, G, 33)])
def test_matvec_double_float_tensor_core(afn, n, d, ker, nrhs):
    # eight or more columns: double-float kernel values, the sum over j exact on the
    # tensor cores (BF16 digits); ragged n, zero-padded last piece, one-point system
    X = inputs.normal_points(n, d, 350 + n)
    P = inputs.rhs(n, nrhs, 351 + n)
    l = 0.7 * np.sqrt(d)
    ref = oracle.matvec(X, ker, l, 1e-2, P)
    bound = scale_bound(X, ker, l, 1e-2, P)
    for prec in (afn.MATVEC_DF_TC, afn.MATVEC_DF_CC):
        q = afn.afn_kernel_matvec(X, ker, l, 1e-2, P, precision=prec)
        err = np.abs(q - ref.reshape(q.shape)) / (bound.reshape(q.shape) + 1e-300)
        assert err.max() <= 1e-12, (prec, err.max())


def test_matvec_double_float_tensor_core_scaled_columns(afn):
    # columns of very different magnitude (each has its own digit exponent) and a zero column
    n = 3000
    X = inputs.normal_points(n, 8, 361)
    P = inputs.rhs(n, 12, 362) * np.array([1e-200, 1e-8, 1.0, 1e6, 1e150, 0.0, 3.0, 1e-3,
                                             7.0, 1e-280, 1e280, 0.5])
    ref = oracle.matvec(X, G, 2.0, 1e-2, P)
    q = afn.afn_kernel_matvec(X, G, 2.0, 1e-2, P, precision=afn.MATVEC_DF_TC)
    bound = scale_bound(X, G, 2.0, 1e-2, P).reshape(q.shape)
    err = np.abs(q - ref.reshape(q.shape)) / (bound + 1e-300)
    assert np.all(q[:, 5] == 0.0)
    assert err.max() <= 1e-12, err.max()


@pytest.mark.parametrize("n,d,ker,nrhs", [(257, 3, G, 1), (1000, 8, M32, 3), (2049, 16, G, 32),
                                          (1500, 2, M32, 7), (1500, 3, M32, 64), (2049, 8, G, 80),
                                          (777, 16, G, 64)])
def test_matvec_fp32(afn, n, d, ker, nrhs):
    # 64-column pieces (and 64 + 16) run the tcgen05 kernel with N = 64
    X = inputs.normal_points(n, d, 400 + n)
    P = inputs.rhs(n, nrhs, 401 + n)
    l = 0.7 * np.sqrt(d)
    q = afn.afn_kernel_matvec(X, ker, l, 1e-2, P, precision=afn.PREC_MIXED)
    ref = oracle.matvec(X, ker, l, 1e-2, P)
    bound = scale_bound(X, ker, l, 1e-2, P).reshape(q.shape)
    err = np.abs(q - ref.reshape(q.shape)) / bound
    assert err.max() <= 2e-5, err.max()


@pytest.mark.parametrize("which", ["normal_8d", "clusters_3d"])
def test_matvec_fp32_tensor_core_full_size(afn, which):
    # the launch configuration the benchmark times (32-column pieces on the tcgen05 kernel):
    # n = 50k, d = 8, Gaussian, 32 columns; n = 200k, d = 3, Matern-3/2, 64 columns
    if which == "normal_8d":
        s = inputs.normal_8d(l=2.0, nrhs=32)
        ker, l, mu = G, 2.0, 1e-2
    else:
        s = inputs.clusters_3d(nrhs=64)
        ker, l, mu = s.kernel, s.l, s.mu
    rows = inputs.rng(11).choice(s.n, 48, replace=False)
    q = afn.afn_kernel_matvec(s.X, ker, l, mu, s.B, precision=afn.PREC_MIXED)
    ref = oracle.matvec_rows(s.X, ker, l, mu, s.B, rows)
    absb = oracle.matvec_rows(s.X, ker, l, mu, np.abs(s.B), rows)
    assert np.all(np.abs(q[rows] - ref) <= 2e-5 * absb)


def test_matvec_sampled_rows_full_size(afn):
    s = inputs.normal_8d(l=2.0, nrhs=2)
    rows = inputs.rng(9).choice(s.n, 64, replace=False)
    for prec, tolr in ((afn.PREC_FP64, 1e-12), (afn.MATVEC_DF, 1e-11), (afn.PREC_MIXED, 2e-5)):
        q = afn.afn_kernel_matvec(s.X, G, 2.0, 1e-2, s.B, precision=prec)
        ref = oracle.matvec_rows(s.X, G, 2.0, 1e-2, s.B, rows)
        absb = oracle.matvec_rows(s.X, G, 2.0, 1e-2, np.abs(s.B), rows)
        assert np.all(np.abs(q[rows] - ref) <= tolr * absb)


def test_matvec_double_float_tensor_core_full_size(afn):
    # the residual replacement of the headline solve: n = 50k, d = 8, 32 columns, the
    # tensor-core double-float matvec, on sampled rows (first and last rows included)
    s = inputs.normal_8d(l=2.0, nrhs=32)
    rows = _sample_rows(s.n, 40, 12, 12)
    q = afn.afn_kernel_matvec(s.X, G, 2.0, 1e-2, s.B, precision=afn.MATVEC_DF_TC)
    ref = oracle.matvec_rows(s.X, G, 2.0, 1e-2, s.B, rows)
    absb = oracle.matvec_rows(s.X, G, 2.0, 1e-2, np.abs(s.B), rows)
    assert np.all(np.abs(q[rows] - ref) <= 1e-11 * absb)


# ---------------------------------------------------------------- build ---
def _cmp(a, b, rtol):
    scale = np.abs(b).max() if b.size else 1.0
    return float(np.abs(a - b).max() / scale) if b.size else 0.0


@pytest.mark.parametrize("n,d,ker,l,mu,k,w", [
    (2000, 3, G, 0.1, 1e-4, 200, 32),      # the n=2000 uniform-cube workload
    (900, 2, M32, 0.15, 1e-3, 90, 20),
    (513, 5, G, 0.6, 1e-2, 64, 7),
    (300, 3, G, 0.2, 1e-3, 0, 10),          # k = 0: FSAI of K + mu I
    (300, 3, M32, 0.2, 1e-3, 300, 10),      # k = n: no Schur rows
    (200, 4, G, 0.3, 1e-2, 33, 1),          # w = 1: diagonal G
    (1400, 3, G, 0.08, 1e-3, 1000, 4),      # k = 1000: batched and ragged blocks at every
                                            # level of the recursive triangular inverse
    (1500, 3, M32, 0.2, 1e-3, 150, 100),    # w = 100 (the paper's FSAI-100): 128-wide tiles
])
def test_build_parity_fp64(afn, n, d, ker, l, mu, k, w):
    X = inputs.uniform_points(n, d, 500 + n)
    ref = oracle.afn_build(X, ker, l, mu, k, w)
    h = afn.afn_build(X, ker, l, mu, k, w, precision=afn.PREC_FP64)
    bi = h.info
    assert (bi.k, bi.nr, bi.w) == (ref["k"], ref["nr"], ref["w"])
    assert np.array_equal(afn.afn_get_perm(h), ref["perm"])
    if ref["k"]:
        assert _cmp(afn.afn_get_L(h), ref["L"], 0) <= 1e-10
    if ref["nr"]:
        pat, Gv = afn.afn_get_G(h)
        assert np.array_equal(pat, ref["pattern"])
        assert _cmp(Gv, ref["G"], 0) <= 1e-10
        if ref["k"]:
            # W^T = K12^T L^{-T}: check against the oracle's L and K12
            W = np.linalg.solve(ref["L"], ref["K12"]).T
            assert _cmp(afn.afn_get_W(h), W, 0) <= 1e-10
    # the apply (Alg. 3) against the oracle's apply on the same input
    r = inputs.rhs(n, 2, 600 + n)
    s_gpu = afn.afn_apply_precond(h, r)
    s_ref = np.stack([oracle.afn_apply(ref, r[:, c]) for c in range(2)], 1)
    assert _cmp(s_gpu, s_ref, 0) <= 1e-8
    afn.afn_free(h)


@pytest.mark.parametrize("n,d,ker,l,mu,k,w", [(2000, 3, G, 0.1, 1e-4, 200, 32),
                                               (900, 2, M32, 0.15, 1e-3, 90, 20),
                                               (1400, 3, G, 0.08, 1e-3, 1000, 4),
                                               (1500, 3, M32, 0.2, 1e-3, 150, 100)])
def test_build_parity_df(afn, n, d, ker, l, mu, k, w):
    # double-float handles: FP64 Cholesky and triangular inverse, W = K21 L^{-T} and the FSAI
    # Gram in double-float arithmetic on the FP32 pipes (about 48-bit accuracy)
    X = inputs.uniform_points(n, d, 500 + n)
    ref = oracle.afn_build(X, ker, l, mu, k, w)
    h = afn.afn_build(X, ker, l, mu, k, w, precision=afn.PREC_DF)
    assert afn.afn_get_build_info(h).precision == afn.PREC_DF
    assert np.array_equal(afn.afn_get_perm(h), ref["perm"])
    assert _cmp(afn.afn_get_L(h), ref["L"], 0) <= 1e-10
    W = np.linalg.solve(ref["L"], ref["K12"]).T
    assert _cmp(afn.afn_get_W(h), W, 0) <= 1e-10
    pat, Gv = afn.afn_get_G(h)
    assert np.array_equal(pat, ref["pattern"])
    assert _cmp(Gv, ref["G"], 0) <= 1e-10
    afn.afn_free(h)


@pytest.mark.parametrize("n,d,ker,l,mu,k,w", [(2000, 3, G, 0.1, 1e-4, 200, 32),
                                               (3001, 8, M32, 2.0, 1e-2, 300, 64)])
def test_build_mixed_fp64_factors(afn, n, d, ker, l, mu, k, w):
    # factors = FP64: a mixed handle's W and G are built as for an FP64 handle (G within
    # the FP64 bar), then rounded to FP32 for the apply
    X = inputs.uniform_points(n, d, 650 + n)
    ref = oracle.afn_build(X, ker, l, mu, k, w)
    h = afn.afn_build(X, ker, l, mu, k, w, precision=afn.PREC_MIXED, factors=afn.FACTORS_FP64)
    assert np.array_equal(afn.afn_get_perm(h), ref["perm"])
    pat, Gv = afn.afn_get_G(h)
    assert np.array_equal(pat, ref["pattern"])
    assert _cmp(Gv, ref["G"], 0) <= 1e-10
    W = np.linalg.solve(ref["L"], ref["K12"]).T
    assert _cmp(afn.afn_get_W(h), W, 0) <= 1e-7          # the FP32 copy of the FP64 W
    r = inputs.rhs(n, 2, 660 + n)
    s_gpu = afn.afn_apply_precond(h, r)
    s_ref = np.stack([oracle.afn_apply(ref, r[:, c]) for c in range(2)], 1)
    err = _cmp(s_gpu, s_ref, 0)
    assert err <= 1e-3, err                                # FP32 apply of the FP64 factors
    afn.afn_free(h)


@pytest.mark.parametrize("ker,d,l,w", [(G, 3, 0.15, 32), (M32, 8, 2.5, 50)])
def test_build_maximin_schur_order(afn, ker, d, l, w):
    # schur_order = 1: the Schur rows in the order FPS continued over all points picks
    # them (the maximin ordering of the screening-effect argument, Sec. 3.1).  The oracle
    # runs the same definition: its full FPS order, then Alg. 2 on the points taken in that
    # order with the first k as landmarks.  FP64: permutation and pattern bit-exact, L and
    # G within 1e-10, iteration counts within +-2
    n, k, mu = 3000, 300, 1e-3
    X = inputs.uniform_points(n, d, 860 + d)
    order = oracle.fps(X, n, 0)
    ref = oracle.afn_build(X[order], ker, l, mu, k, w, landmarks=np.arange(k))
    h = afn.afn_build(X, ker, l, mu, k, w, precision=afn.PREC_FP64, schur_order=1)
    assert np.array_equal(afn.afn_get_perm(h), order)
    pat, Gv = afn.afn_get_G(h)
    assert np.array_equal(pat, ref["pattern"])
    assert _cmp(afn.afn_get_L(h), ref["L"], 0) <= 1e-10
    assert _cmp(Gv, ref["G"], 0) <= 1e-10
    b = inputs.rhs(n, 1, 870 + d)
    xr, itr, relr, st_ = oracle.pcg(ref, b[order, 0], 1e-6)
    x, info = afn.afn_solve(h, b, 1e-6)
    assert abs(int(info["iters"][0]) - itr) <= 2, (info["iters"], itr)
    assert oracle.true_relres(X, ker, l, mu, x, b).max() <= 1e-6
    afn.afn_free(h)
    with pytest.raises(afn.AfnError) as e:
        afn.afn_build(X, ker, l, mu, k, w, precision=afn.PREC_FP64, schur_order=1,
                      landmarks=afn.LM_UNIFORM)
    assert e.value.status == afn.AFN_ERR_ARG


@pytest.mark.parametrize("w", [24, 100])
def test_build_mixed_close_to_oracle(afn, w):
    # w = 100: the FP32 FSAI build with the 128-wide Schur blocks
    X = inputs.uniform_points(1200, 3, 700)
    ref = oracle.afn_build(X, G, 0.1, 1e-3, 120, w)
    h = afn.afn_build(X, G, 0.1, 1e-3, 120, w, precision=afn.PREC_MIXED)
    assert np.array_equal(afn.afn_get_perm(h), ref["perm"])
    pat, Gv = afn.afn_get_G(h)
    assert np.array_equal(pat, ref["pattern"])
    assert _cmp(afn.afn_get_L(h), ref["L"], 0) <= 1e-10      # Cholesky stays FP64
    assert _cmp(Gv, ref["G"], 0) <= 1e-2                      # FP32 Schur blocks
    # W^T = K21 L^{-T} from the FP32 kernel block and the triangular inverse (FP64, rounded)
    W = np.linalg.solve(ref["L"], ref["K12"]).T
    errw = _cmp(afn.afn_get_W(h), W, 0)
    assert errw <= 1e-3, errw


@pytest.mark.parametrize("n,k,nrhs", [(3001, 300, 32), (2600, 130, 16), (3001, 300, 48)])
def test_mixed_apply_tensor_core_products(afn, n, k, nrhs):
    # the FP32 apply of a mixed handle with the W products on the tcgen05
    # tensor cores (three-pass tf32, option apply_tc) against the same apply on the CUDA
    # cores and against the oracle's FP64 apply of the oracle's own build; ragged k
    # and n - k (not multiples of the 32-element stages or 128-row tiles)
    X = inputs.normal_points(n, 8, 800 + n)
    h_tc = afn.afn_build(X, G, 1.0, 1e-2, k, 32, precision=afn.PREC_MIXED, apply_tc=1)
    h_cc = afn.afn_build(X, G, 1.0, 1e-2, k, 32, precision=afn.PREC_MIXED, apply_tc=0)
    bi = h_tc.info
    assert bi.k == k and bi.nr == n - k
    r = inputs.rhs(n, nrhs, 900 + n)
    before = afn.afn_get_build_info(h_tc).device_bytes
    s_tc = afn.afn_apply_precond(h_tc, r)
    grown = afn.afn_get_build_info(h_tc).device_bytes - before
    assert grown >= 2 * 4 * k * (n - k)            # the two tiled images of W were built
    s_cc = afn.afn_apply_precond(h_cc, r)
    assert np.all(np.isfinite(s_tc))
    assert _cmp(s_tc, s_cc, 0) <= 2e-5
    # FP32 apply of an FP32-built preconditioner against the FP64 oracle
    ref = oracle.afn_build(X, G, 1.0, 1e-2, k, 32)
    s_ref = np.stack([oracle.afn_apply(ref, r[:, c]) for c in range(3)], 1)
    assert _cmp(s_tc[:, :3], s_ref, 0) <= 1e-2
    afn.afn_free(h_tc)
    afn.afn_free(h_cc)


def _bf16(a):
    """Round FP64 values to BF16 (8-bit significand, round to nearest even) via FP32."""
    f = np.asarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    f = (f + 0x7FFF + ((f >> 16) & 1)) & 0xFFFF0000
    return f.astype(np.uint32).view(np.float32).astype(np.float64)


def _apply_wform(Lo, Wt, pat, Gv, r):
    """Alg. 3 in the W form, FP64: z' = L^{-1} r1, t = r2 - W^T z', s2 = G^T G t,
    s1 = L^{-T} (z' - W s2); Wt is W^T (nr x k), G as ELL (pattern, values)."""
    k, nr = Lo.shape[0], Wt.shape[0]
    Gd = np.zeros((nr, nr))
    for i in range(nr):
        for p_, c in enumerate(pat[i]):
            if c >= 0:
                Gd[i, c] = Gv[i, p_]
    zp = np.linalg.solve(Lo, r[:k])
    t = r[k:] - Wt @ zp
    s2 = Gd.T @ (Gd @ t)
    s1 = np.linalg.solve(Lo.T, zp - Wt.T @ s2)
    return np.concatenate([s1, s2])


@pytest.mark.parametrize("n,k,nrhs", [(3001, 300, 64), (2600, 130, 16), (3001, 300, 80),
                                      (2200, 700, 32)])
def test_mixed_apply_bf16_tensor_core_products(afn, n, k, nrhs):
    # apply_tc = 2: the W products on the tcgen05 tensor cores with a BF16 copy of W and the
    # vectors in three BF16 terms.  Against the same apply written out in FP64 with the
    # handle's own factors and W rounded to BF16 (the only approximation besides FP32
    # arithmetic); ragged k and n - k, 16/32/64-column pieces
    X = inputs.normal_points(n, 8, 830 + n)
    h = afn.afn_build(X, G, 1.0, 1e-2, k, 32, precision=afn.PREC_MIXED, apply_tc=2)
    bi = h.info
    assert bi.k == k and bi.nr == n - k
    r = inputs.rhs(n, nrhs, 840 + n)
    before = afn.afn_get_build_info(h).device_bytes
    s_tc = afn.afn_apply_precond(h, r)
    grown = afn.afn_get_build_info(h).device_bytes - before
    assert grown >= 2 * 2 * k * (n - k)            # the two BF16 images of W were built
    Lo = afn.afn_get_L(h)
    Wt = afn.afn_get_W(h)
    pat, Gv = afn.afn_get_G(h)
    Gv32 = Gv.astype(np.float32).astype(np.float64)
    cols = [0, nrhs // 2, nrhs - 1]
    ref = np.stack([_apply_wform(Lo, _bf16(Wt), pat, Gv32, r[:, c]) for c in cols], 1)
    err = _cmp(s_tc[:, cols], ref, 0)
    assert err <= 1e-3, err
    afn.afn_free(h)


def test_not_spd_reported(afn):
    # duplicated landmarks make K11 singular; mu tiny keeps K11 + mu I at the
    # edge -- with mu = 1e-300 the Cholesky pivot underflows to <= 0
    X = np.zeros((20, 3))
    with pytest.raises(afn.AfnError) as e:
        afn.afn_build(X, G, 1.0, 1e-300, 5, 4, landmarks=afn.LM_UNIFORM)
    assert e.value.status == afn.AFN_ERR_NOT_SPD


def test_nan_input_rejected(afn):
    X = inputs.uniform_points(50, 3, 1)
    X[7, 1] = np.nan
    with pytest.raises(afn.AfnError) as e:
        afn.afn_build(X, G, 0.3, 1e-3, 5, 4)
    assert e.value.status == afn.AFN_ERR_ARG


# ---------------------------------------------------------------- solve ---
def test_solve_fp64_uniform_cube(afn):
    s = inputs.uniform_cube_3d()
    ref = oracle.afn_build(s.X, s.kernel, s.l, s.mu, s.k, s.w)
    xr, itr, relr, str_ = oracle.pcg(ref, s.B[:, 0], 1e-6)
    h = afn.afn_build(s.X, s.kernel, s.l, s.mu, s.k, s.w, precision=afn.PREC_FP64)
    x, info = afn.afn_solve(h, s.B, 1e-6)
    rel = oracle.true_relres(s.X, s.kernel, s.l, s.mu, x, s.B)
    assert rel.max() <= 1e-6
    assert abs(int(info["iters"][0]) - itr) <= 2, (info["iters"], itr)
    assert np.linalg.norm(x[:, 0] - xr) / np.linalg.norm(xr) <= 1e-4
    afn.afn_free(h)


def test_solve_df_uniform_cube(afn):
    """The DF precision (FP64 PCG, factors and apply; double-float matvec on
    the FP32 pipes) follows the FP64 oracle like the FP64 path: residual <=
    tol, iterations within +-2."""
    s = inputs.uniform_cube_3d()
    ref = oracle.afn_build(s.X, s.kernel, s.l, s.mu, s.k, s.w)
    xr, itr, relr, str_ = oracle.pcg(ref, s.B[:, 0], 1e-6)
    h = afn.afn_build(s.X, s.kernel, s.l, s.mu, s.k, s.w, precision=afn.PREC_DF)
    assert afn.afn_get_build_info(h).precision == afn.PREC_DF
    x, info = afn.afn_solve(h, s.B, 1e-6)
    rel = oracle.true_relres(s.X, s.kernel, s.l, s.mu, x, s.B)
    assert rel.max() <= 1e-6
    assert abs(int(info["iters"][0]) - itr) <= 2, (info["iters"], itr)
    afn.afn_free(h)


@pytest.mark.parametrize("ker,nrhs", [(G, 1), (M32, 5), (G, 33)])
def test_solve_fp64_and_mixed_multi_rhs(afn, ker, nrhs):
    X = inputs.uniform_points(1500, 3, 800 + nrhs)
    B = inputs.rhs(1500, nrhs, 801 + nrhs)
    B[:, 0] *= 1e3
    if nrhs > 1:
        B[:, 1] = 0.0                        # a zero column: x = 0, converged at once
    l, mu, k, w, tol = 0.12, 1e-3, 150, 24, 1e-6
    ref = oracle.afn_build(X, ker, l, mu, k, w)
    xr, itr, relr, str_ = oracle.pcg(ref, B[:, 0], tol)
    for prec in (afn.PREC_FP64, afn.PREC_MIXED):
        h = afn.afn_build(X, ker, l, mu, k, w, precision=prec)
        x, info = afn.afn_solve(h, B, tol)
        assert info["status"] == afn.AFN_OK
        rel = oracle.true_relres(X, ker, l, mu, x, B + (B == 0) * 0)
        rel = np.where(np.linalg.norm(B, axis=0) > 0, rel, 0.0)
        assert np.nanmax(rel) <= tol, (prec, rel)
        if nrhs > 1:
            assert np.all(x[:, 1] == 0.0)
        if prec == afn.PREC_FP64:
            assert abs(int(info["iters"][0]) - itr) <= 2
        afn.afn_free(h)


def test_solve_mixed_flexible_pcg(afn):
    # flexible PCG (Polak-Ribiere beta) on a mixed handle reaches tol as recomputed by the
    # oracle, with iteration counts close to the textbook form's
    X = inputs.uniform_points(2500, 3, 820)
    B = inputs.rhs(2500, 16, 821)
    its = {}
    for flex in (0, 1):
        h = afn.afn_build(X, G, 0.1, 1e-3, 250, 32, precision=afn.PREC_MIXED, flexible=flex)
        x, info = afn.afn_solve(h, B, 1e-6)
        assert info["converged"] == 16
        rel = oracle.true_relres(X, G, 0.1, 1e-3, x[:, :3], B[:, :3])
        assert np.all(rel <= 1e-6), rel
        its[flex] = int(info["iters"].max())
        afn.afn_free(h)
    assert abs(its[1] - its[0]) <= max(4, its[0] // 10), its


def test_solve_k_equals_n_one_iteration(afn):
    X = inputs.uniform_points(150, 2, 900)
    b = inputs.rhs(150, 1, 901)
    h = afn.afn_build(X, G, 0.3, 1e-2, 150, 8, precision=afn.PREC_FP64)
    x, info = afn.afn_solve(h, b, 1e-10)
    assert info["iters"][0] == 1
    a = oracle.dense_solve(X, G, 0.3, 1e-2, b[:, 0])
    assert np.linalg.norm(x[:, 0] - a) / np.linalg.norm(a) < 1e-8


def test_solve_device_pointers(afn):
    torch = pytest.importorskip("torch")
    X = inputs.uniform_points(800, 3, 950)
    B = inputs.rhs(800, 3, 951)
    h = afn.afn_build(torch.tensor(X, device="cuda"), G, 0.15, 1e-3, 80, 16,
                      precision=afn.PREC_MIXED)
    x, info = afn.afn_solve(h, torch.tensor(B, device="cuda"), 1e-6)
    assert x.is_cuda
    rel = oracle.true_relres(X, G, 0.15, 1e-3, x.cpu().numpy(), B)
    assert rel.max() <= 1e-6


def test_solve_headline_normal_8d_oracle_residual(afn):
    # the benchmark's system (n = 50k, d = 8, Gaussian l = 1, mu = 1e-2, Alg. 4 k capped at
    # 4000, w = 64, 32 right-hand sides, mixed precision, tol 1e-6): the true relative
    # residual of two columns recomputed by the oracle's FP64 matvec
    s = inputs.normal_8d(l=1.0, nrhs=32)
    h = afn.afn_build(s.X, G, 1.0, 1e-2, 4000, 64, precision=afn.PREC_MIXED,
                      rank_mode=afn.RANK_ESTIMATE, rank_subsample=1000, seed=s.seed,
                      max_iter=3000)
    x, info = afn.afn_solve(h, s.B, 1e-6)
    assert info["converged"] == 32, info
    cols = [0, 31]
    rel = oracle.true_relres(s.X, G, 1.0, 1e-2, x[:, cols], s.B[:, cols])
    assert np.all(rel <= 1e-6), rel
    # the library's own FP64 residual agrees with the oracle's
    assert np.allclose(info["relres"][cols], rel, rtol=1e-3, atol=1e-12)
    afn.afn_free(h)


def test_solve_clusters_3d_prefix_bf16_oracle_residual(afn):
    # the n = 200k, d = 3 clustered workload's configuration (Matern-3/2 l = 0.05, mu = 1e-3,
    # w = 50, 64 right-hand sides, BF16 tensor-core W products, FP64 residual replacements)
    # on its first 50,000 points with the same k / n (500 landmarks): the true relative
    # residual of two columns recomputed by the oracle in FP64
    s = inputs.clusters_3d(nrhs=64)
    n, k = 50_000, 500
    X, B = s.X[:n], np.asfortranarray(s.B[:n])
    h = afn.afn_build(X, s.kernel, s.l, s.mu, k, s.w, precision=afn.PREC_MIXED, apply_tc=2,
                      max_iter=3000)
    x, info = afn.afn_solve(h, B, 1e-6)
    assert info["converged"] == 64, info
    cols = [0, 63]
    rel = oracle.true_relres(X, s.kernel, s.l, s.mu, x[:, cols], B[:, cols])
    assert np.all(rel <= 1e-6), rel
    afn.afn_free(h)


def test_solve_clusters_3d_full_size_bf16(afn):
    # the full n = 200k clustered workload (k = 2000): every column's residual recomputed by
    # the FP64-accurate double-float matvec (parity-tested against the oracle), and that
    # matvec checked against the oracle on sampled rows of the solution
    s = inputs.clusters_3d(nrhs=64)
    h = afn.afn_build(s.X, s.kernel, s.l, s.mu, s.k, s.w, precision=afn.PREC_MIXED, apply_tc=2,
                      max_iter=3000)
    x, info = afn.afn_solve(h, s.B, 1e-6)
    assert info["converged"] == 64, info
    q = afn.afn_kernel_matvec(s.X, s.kernel, s.l, s.mu, x, precision=afn.MATVEC_DF)
    rel = np.linalg.norm(s.B - q, axis=0) / np.linalg.norm(s.B, axis=0)
    assert np.all(rel <= 1e-6), rel.max()
    rows = _sample_rows(s.n, 50, 41, 24)
    cols = [0, 63]
    ref = oracle.matvec_rows(s.X, s.kernel, s.l, s.mu, x[:, cols], rows)
    absb = oracle.matvec_rows(s.X, s.kernel, s.l, s.mu, np.abs(x[:, cols]), rows)
    assert np.all(np.abs(q[np.ix_(rows, cols)] - ref) <= 1e-11 * absb)
    afn.afn_free(h)


# ------------------------------------------------------------- Alg. 4 ---
@pytest.mark.parametrize("l,n,m", [(0.05, 3000, 120), (0.3, 3000, 120), (1.0, 3000, 150),
                                   (3.0, 800, 200)])
def test_rank_estimate_parity(afn, l, n, m):
    X = inputs.uniform_points(n, 3, 35)
    kg = afn.afn_rank_estimate(X, G, l, 1e-2, m=m, seed=7, k_max=100000)
    ko = oracle.rank_estimate(X, G, l, 1e-2, m=m, seed=7, k_max=100000)
    assert kg == ko


def test_rank_estimate_normal_8d_full(afn):
    s = inputs.normal_8d(l=2.0, nrhs=1)
    kg = afn.afn_rank_estimate(s.X, G, 2.0, 1e-2, m=1000, seed=s.seed, k_max=4000)
    ko = oracle.rank_estimate(s.X, G, 2.0, 1e-2, m=1000, seed=s.seed, k_max=4000)
    assert kg == ko


# ------------------------------------------------------ Nystrom branch ---
NYS = 1   # afn.PRECOND_NYSTROM


@pytest.mark.parametrize("n,d,ker,l,mu,k", [(600, 3, G, 0.4, 1e-2, 60), (900, 2, M32, 0.5, 1e-3, 45),
                                            (500, 5, G, 1.5, 1e-2, 0)])
def test_nystrom_apply_parity(afn, n, d, ker, l, mu, k):
    # eq. (nystrom1-smw): the GPU applies (K_nys + mu I)^{-1} through the SMW identity with a
    # Cholesky of mu I + B^T B; the oracle literally, with an eigendecomposition
    X = inputs.uniform_points(n, d, 1100 + n)
    h = afn.afn_build(X, ker, l, mu, k, 16, precision=afn.PREC_FP64, precond=NYS)
    assert h.info.precond == NYS and h.info.k == k
    ref = oracle.nystrom_build(X, ker, l, mu, k)
    assert np.array_equal(afn.afn_get_perm(h), ref["perm"])
    r = inputs.rhs(n, 3, 1200 + n)
    s_gpu = afn.afn_apply_precond(h, r)
    s_ref = np.stack([oracle.nystrom_apply(ref, r[:, c]) for c in range(3)], 1)
    assert _cmp(s_gpu, s_ref, 0) <= 1e-9
    afn.afn_free(h)


def test_nystrom_solve_iterations_match_oracle(afn):
    X = inputs.uniform_points(1500, 3, 1300)
    b = inputs.rhs(1500, 1, 1301)[:, 0]
    ref = oracle.nystrom_build(X, G, 0.3, 1e-2, 100)
    _, it_ref, rel_ref, st_ref = oracle.pcg_nystrom(ref, b, 1e-6, max_iter=500)
    assert st_ref == 0
    h = afn.afn_build(X, G, 0.3, 1e-2, 100, 16, precision=afn.PREC_FP64, precond=NYS, max_iter=500)
    x, info = afn.afn_solve(h, b, 1e-6)
    assert info["converged"] == 1
    assert abs(int(info["iters"][0]) - it_ref) <= 2
    assert oracle.true_relres(X, G, 0.3, 1e-2, x, b) <= 1e-6
    afn.afn_free(h)


def test_nystrom_mixed_multi_rhs_reaches_tol(afn):
    X = inputs.normal_points(4000, 8, 1400)
    B = inputs.rhs(4000, 32, 1401)
    h = afn.afn_build(X, G, 4.0, 1e-2, 300, 32, precision=afn.PREC_MIXED, precond=NYS, max_iter=3000)
    x, info = afn.afn_solve(h, B, 1e-6)
    assert info["converged"] == 32
    rel = oracle.true_relres(X, G, 4.0, 1e-2, x[:, :2], B[:, :2])
    assert np.all(rel <= 1e-6)
    afn.afn_free(h)


def test_alg5_strategy_branch(afn):
    # Alg. 5: the branch follows the Alg. 4 estimate against the threshold, as in the oracle
    X = inputs.uniform_points(3000, 3, 1500)
    k = oracle.rank_estimate(X, G, 0.5, 1e-2, m=200, seed=7, k_max=3000)[0]
    for thr, want in ((k + 1, NYS), (k, 0)):
        h = afn.afn_build(X, G, 0.5, 1e-2, 3000, 16, precision=afn.PREC_FP64,
                          precond=afn.PRECOND_AUTO, precond_threshold=thr, rank_subsample=200,
                          seed=7)
        assert h.info.k == k and h.info.precond == want
        afn.afn_free(h)
    with pytest.raises(afn.AfnError) as e:
        afn.afn_build_batched([dict(points=X[:300], kernel=G, l=0.5, mu=1e-2, k_max=30,
                                    fsai_nnz=8)], precond=NYS)
    assert e.value.status == afn.AFN_ERR_ARG
