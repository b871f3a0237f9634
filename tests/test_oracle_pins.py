"""Pins for the FP64 CPU oracle (no GPU).

Each test checks the oracle against something other than itself: closed
forms, brute force on tiny inputs, invariants the paper states or implies,
and special cases that reduce to a textbook/library routine.  A plausible
slip in the oracle (a dropped mu, l^2 vs 2 l^2, a transposed K12, a wrong
tie-break, a missing square root in FSAI) fails at least one of them.
"""
import itertools
import math

import numpy as np
import pytest

import oracle
from paper_2304_05460_gb300 import inputs

G, M32 = oracle.GAUSSIAN, oracle.MATERN32


def pts(n, d, seed, scale=1.0):
    return inputs.uniform_points(n, d, seed) * scale


# ---------------------------------------------------------------- kernels ---
def test_kernel_closed_forms():
    # eq. (gaussianf): exp(-r^2 / l^2); at r = l the value is e^-1 (not e^-1/2)
    x = np.array([0.0, 0.0, 0.0])
    y = np.array([0.3, 0.0, 0.4])          # r = 0.5 exactly
    K = oracle.kernel_matrix(x[None], y[None], G, 0.5)[0, 0]
    assert K == pytest.approx(0.36787944117144233, rel=1e-15)
    assert oracle.kernel_matrix(x[None], y[None], G, 0.25)[0, 0] == pytest.approx(math.exp(-4.0), rel=1e-15)
    # Matern-3/2 (Sec. 5): (1 + sqrt3 r/l) exp(-sqrt3 r/l); r = l gives (1+sqrt3) e^-sqrt3
    Km = oracle.kernel_matrix(x[None], y[None], M32, 0.5)[0, 0]
    assert Km == pytest.approx((1 + math.sqrt(3)) * math.exp(-math.sqrt(3)), rel=1e-15)
    assert Km == pytest.approx(0.4833577245965077, rel=1e-13)
    # r = 0 gives 1 for both
    X = pts(7, 3, 1)
    for ker in (G, M32):
        Kxx = oracle.kernel_matrix(X, X, ker, 0.3)
        assert np.all(np.diag(Kxx) == 1.0)
        assert np.array_equal(Kxx, Kxx.T)
        assert np.all((Kxx > 0) & (Kxx <= 1))


def test_kernel_rescale_invariance_bitwise():
    # Remark after Thm 4.1: length-scale l acts as a rescaling x/l of the points
    X = pts(20, 3, 2)
    for ker in (G, M32):
        a = oracle.kernel_matrix(X, X, ker, 0.3)
        b = oracle.kernel_matrix(4.0 * X, 4.0 * X, ker, 1.2)
        assert np.array_equal(a, b)


def test_kernel_spsd():
    X = pts(60, 2, 3)
    for ker in (G, M32):
        ev = np.linalg.eigvalsh(oracle.kernel_matrix(X, X, ker, 0.2))
        assert ev.min() > -1e-12


def test_matvec_matches_dense_product():
    X = pts(50, 3, 4)
    P = inputs.rhs(50, 3, 5)
    for ker in (G, M32):
        K = oracle.kernel_matrix(X, X, ker, 0.2)
        ref = K @ P + 0.01 * P
        out = oracle.matvec(X, ker, 0.2, 0.01, P)
        assert np.allclose(out, ref, rtol=1e-13, atol=1e-13)


# -------------------------------------------------------------------- FPS ---
def _min_dists(X, S):
    D = np.sqrt(((X[:, None, :] - X[None, S, :]) ** 2).sum(-1))
    return D.min(1)


def test_fps_brute_force_each_step():
    # Alg. 6 / Sec. 4: at step i+1 pick argmax_{x not in X_i} dist(x, X_i)
    for seed, (n, d, k) in enumerate([(40, 2, 15), (33, 3, 33), (25, 5, 10)]):
        X = pts(n, d, 10 + seed)
        idx = oracle.fps(X, k, start=3)
        assert idx[0] == 3
        assert len(set(idx.tolist())) == k
        for i in range(1, k):
            md = _min_dists(X, list(idx[:i]))
            md[list(idx[:i])] = -1
            assert idx[i] == int(np.argmax(md))


def test_fps_tie_break_lowest_index():
    X = np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0], [1.0, 1.0]])
    assert oracle.fps(X, 4, 0).tolist() == [0, 3, 1, 2]
    # duplicated points: never selected twice, all indices appear for k = n
    Y = np.array([[0.0, 0.0], [0.0, 0.0], [1.0, 0.0], [1.0, 0.0], [0.5, 0.5]])
    s = oracle.fps(Y, 5, 0)
    assert sorted(s.tolist()) == [0, 1, 2, 3, 4]
    assert s.tolist() == [0, 2, 4, 1, 3]


def _fill_sep(X, S):
    h = _min_dists(X, S).max()
    D = np.sqrt(((X[S][:, None] - X[S][None]) ** 2).sum(-1))
    q = D[np.triu_indices(len(S), 1)].min()
    return h, q


def test_fps_theorem3_invariants():
    # Thm 3: h_{X_k} <= q_{X_k}; in its proof q_{X_{k+1}} >= h_{X_k}
    X = pts(300, 2, 11)
    idx = oracle.fps(X, 40, 0)
    for k in range(2, 40):
        h, q = _fill_sep(X, list(idx[:k]))
        assert h <= q + 1e-15
        _, q1 = _fill_sep(X, list(idx[: k + 1]))
        assert q1 >= h - 1e-15


def test_fps_near_optimality_brute_force():
    # Thm 3: h_{X_k} <= 2 h*  and  q_{X_k} >= q*/2 (optimum by enumeration)
    X = pts(11, 2, 12)
    k = 4
    idx = list(oracle.fps(X, k, 0))
    h, q = _fill_sep(X, idx)
    hs, qs = [], []
    for S in itertools.combinations(range(11), k):
        a, b = _fill_sep(X, list(S))
        hs.append(a)
        qs.append(b)
    assert h <= 2 * min(hs) + 1e-15
    assert q >= max(qs) / 2 - 1e-15


def test_fps_centroid_start():
    X = pts(57, 3, 13)
    c = X.mean(0)
    assert oracle.fps_centroid_start(X) == int(np.argmin(((X - c) ** 2).sum(1)))


def test_fps_rescale_invariance():
    X = pts(200, 3, 14)
    assert np.array_equal(oracle.fps(X, 30, 5), oracle.fps(X * 8.0, 30, 5))


# --------------------------------------------------------- uniform sampler ---
def test_splitmix64_published_vector():
    # SplitMix64 (Steele, Lea, Flood 2014) seeded with 0: first outputs
    s = oracle.splitmix64_stream(0, 3)
    assert [int(v) for v in s] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_uniform_sample_is_partial_fisher_yates():
    n = 1000
    first = int(oracle.splitmix64_stream(12345, 1)[0])
    idx = oracle.uniform_sample(n, 50, 12345)
    assert idx[0] == first % n
    assert len(set(idx.tolist())) == 50 and idx.min() >= 0 and idx.max() < n
    allp = oracle.uniform_sample(37, 37, 9)
    assert sorted(allp.tolist()) == list(range(37))


def test_permutation_landmarks_first():
    lm = np.array([7, 2, 9])
    perm = oracle.permutation(12, lm)
    assert perm.tolist() == [7, 2, 9, 0, 1, 3, 4, 5, 6, 8, 10, 11]


# -------------------------------------------------------------------- KNN ---
def _knn_brute(Xr, w):
    nr = Xr.shape[0]
    out = []
    for i in range(nr):
        j = np.arange(i)
        r2 = ((Xr[:i] - Xr[i]) ** 2).sum(1)
        o = np.lexsort((j, r2))[: w - 1]
        out.append(list(j[o]) + [i])
    return out


@pytest.mark.parametrize("w", [1, 2, 5, 9])
def test_knn_pattern_brute_force(w):
    Xr = pts(70, 3, 15)
    pat, rl = oracle.knn_pattern(Xr, w)
    ref = _knn_brute(Xr, w)
    for i in range(70):
        assert rl[i] == len(ref[i])
        assert pat[i, : rl[i]].tolist() == ref[i]
        assert np.all(pat[i, rl[i]:] == -1)


def test_knn_pattern_ties_on_lattice():
    # integer lattice: many exact distance ties -> lower index first
    g = np.stack(np.meshgrid(np.arange(5.0), np.arange(5.0), indexing="ij"), -1).reshape(-1, 2)
    Xr = g[inputs.rng(16).permutation(25)]
    pat, rl = oracle.knn_pattern(Xr, 6)
    ref = _knn_brute(Xr, 6)
    for i in range(25):
        assert pat[i, : rl[i]].tolist() == ref[i]


# --------------------------------------------------------------- Cholesky ---
def test_cholesky_closed_form_2x2_and_library():
    a, b, c = 4.0, 2.0, 5.0
    Lo = oracle.cholesky(np.array([[a, b], [b, c]]))
    assert np.allclose(Lo, [[2.0, 0.0], [1.0, 2.0]], rtol=0, atol=1e-15)
    X = pts(120, 3, 17)
    A = oracle.kernel_matrix(X, X, G, 0.3) + 1e-3 * np.eye(120)
    Lo = oracle.cholesky(A)
    assert np.allclose(Lo @ Lo.T, A, rtol=0, atol=1e-13)
    assert np.allclose(Lo, np.linalg.cholesky(A), rtol=1e-10, atol=1e-12)
    with pytest.raises(np.linalg.LinAlgError):
        oracle.cholesky(np.array([[1.0, 2.0], [2.0, 1.0]]))


# ------------------------------------------------------------------- FSAI ---
def test_fsai_row_closed_forms():
    assert oracle.fsai_row(np.array([[4.0]]))[0] == pytest.approx(0.5)
    a, b, c = 3.0, 1.0, 2.0
    g = oracle.fsai_row(np.array([[a, b], [b, c]]))
    den = math.sqrt(a * (a * c - b * b))
    assert np.allclose(g, [-b / den, a / den], rtol=1e-14)


def _schur_dense(f):
    """S = K22 + mu I - K12^T (K11 + mu I)^{-1} K12 by numpy (library solve)."""
    Xp, k = f["Xp"], f["k"]
    K = oracle.kernel_matrix(Xp, Xp, f["kernel"], f["l"])
    A = K + f["mu"] * np.eye(len(Xp))
    if k == 0:
        return A[k:, k:]
    return A[k:, k:] - A[:k, k:].T @ np.linalg.solve(A[:k, :k], A[:k, k:])


def _dense_G(f):
    nr, w = f["nr"], f["w"]
    Gd = np.zeros((nr, nr))
    for i in range(nr):
        for p in range(w):
            c = f["pattern"][i, p]
            if c >= 0:
                Gd[i, c] = f["G"][i, p]
    return Gd


@pytest.mark.parametrize("ker,k,w", [(G, 20, 6), (M32, 15, 8), (G, 0, 5), (G, 59, 4)])
def test_fsai_normal_equations_on_schur(ker, k, w):
    # Alg. 1 on S (Sec. 3.1/3.2): (S[s,s] g^T)_j = 0 for j < last; g_last (S g)_last = 1
    X = pts(90, 2, 18)
    f = oracle.afn_build(X, ker, 0.25, 1e-3, k, w)
    S = _schur_dense(f)
    for i in range(f["nr"]):
        m = f["rowlen"][i]
        s = f["pattern"][i, :m]
        g = f["G"][i, :m]
        Sg = S[np.ix_(s, s)] @ g
        assert s[-1] == i
        assert np.allclose(Sg[:-1], 0.0, atol=1e-9 * np.abs(S).max())
        assert g[-1] * Sg[-1] == pytest.approx(1.0, rel=1e-9)
    Gd = _dense_G(f)
    assert np.allclose(np.diag(Gd @ S @ Gd.T), 1.0, rtol=1e-9)
    assert np.allclose(np.triu(Gd, 1), 0.0)


def test_build_uses_landmark_order_and_regularized_k11():
    X = pts(80, 3, 19)
    f = oracle.afn_build(X, G, 0.3, 1e-2, 12, 5)
    assert np.array_equal(f["perm"][:12], oracle.fps(X, 12, 0))
    A11 = oracle.kernel_matrix(X[f["perm"][:12]], X[f["perm"][:12]], G, 0.3) + 1e-2 * np.eye(12)
    assert np.allclose(f["L"] @ f["L"].T, A11, atol=1e-13)
    assert np.array_equal(f["K12"], oracle.kernel_matrix(X[f["perm"][:12]], X[f["perm"][12:]], G, 0.3))


# ---------------------------------------------------------------------- M ---
@pytest.mark.parametrize("ker", [G, M32])
def test_M_two_forms_agree_and_spd(ker):
    # eq. (factorized-form) == eq. (realM); M symmetric positive definite
    X = pts(70, 2, 20)
    f = oracle.afn_build(X, ker, 0.3, 1e-3, 14, 5)
    Mf = oracle.dense_M_factored(f)
    Me = oracle.dense_M_expanded(f)
    assert np.allclose(Mf, Me, rtol=1e-9, atol=1e-9 * np.abs(Me).max())
    assert np.allclose(Mf, Mf.T, atol=1e-10 * np.abs(Mf).max())
    assert np.linalg.eigvalsh(0.5 * (Mf + Mf.T)).min() > 0
    # the (1,1) and (1,2) blocks are exactly those of K + mu I
    K = oracle.kernel_matrix(f["Xp"], f["Xp"], ker, 0.3) + 1e-3 * np.eye(70)
    assert np.allclose(Me[:14, :], K[:14, :], atol=1e-15)


def test_M_exact_with_full_pattern():
    # Sec. 3.2: G^T G = S^{-1} exactly  =>  M = K + mu I
    X = pts(40, 2, 21)
    f = oracle.afn_build(X, G, 0.3, 1e-2, 8, 40)
    K = oracle.kernel_matrix(f["Xp"], f["Xp"], G, 0.3) + 1e-2 * np.eye(40)
    assert np.allclose(oracle.dense_M_factored(f), K, atol=1e-9)
    Gd = _dense_G(f)
    assert np.allclose(Gd.T @ Gd, np.linalg.inv(_schur_dense(f)), rtol=1e-7, atol=1e-7)


def test_M_special_cases_k0_and_kn():
    X = pts(35, 2, 22)
    f0 = oracle.afn_build(X, M32, 0.2, 1e-2, 0, 6)          # pure FSAI of K + mu I
    Gd = _dense_G(f0)
    assert np.allclose(oracle.dense_M_factored(f0), np.linalg.inv(Gd.T @ Gd), rtol=1e-8, atol=1e-9)
    fn = oracle.afn_build(X, M32, 0.2, 1e-2, 35, 6)         # all points landmarks
    K = oracle.kernel_matrix(fn["Xp"], fn["Xp"], M32, 0.2) + 1e-2 * np.eye(35)
    r = inputs.rhs(35, 1, 23)[:, 0]
    assert np.allclose(oracle.afn_apply(fn, r), np.linalg.solve(K, r), rtol=1e-10)


@pytest.mark.parametrize("k,w", [(10, 4), (0, 3), (25, 7)])
def test_apply_inverts_M(k, w):
    # Alg. 3 returns s with M s = r
    X = pts(60, 3, 24)
    f = oracle.afn_build(X, G, 0.35, 1e-3, k, w)
    M = oracle.dense_M_expanded(f)
    r = inputs.rhs(60, 1, 25)[:, 0]
    s = oracle.afn_apply(f, r)
    assert np.allclose(M @ s, r, rtol=1e-8, atol=1e-8 * np.abs(r).max())


def test_build_rescale_invariance_bitwise():
    X = pts(120, 3, 26)
    a = oracle.afn_build(X, M32, 0.2, 1e-3, 20, 6)
    b = oracle.afn_build(4.0 * X, M32, 0.8, 1e-3, 20, 6)
    for key in ("perm", "pattern", "L", "K12", "G"):
        assert np.array_equal(a[key], b[key]), key


# -------------------------------------------------------------------- PCG ---
def test_pcg_reaches_dense_solution():
    X = pts(400, 3, 27)
    b = inputs.rhs(400, 1, 28)[:, 0]
    f = oracle.afn_build(X, G, 0.1, 1e-4, 40, 10)
    x, it, rel, st = oracle.pcg(f, b, 1e-8)
    a = oracle.dense_solve(X, G, 0.1, 1e-4, b)
    assert st == 0 and rel <= 1e-8
    assert np.linalg.norm(x - a) / np.linalg.norm(a) < 1e-4
    r = b - (oracle.kernel_matrix(X, X, G, 0.1) @ x + 1e-4 * x)
    assert np.linalg.norm(r) / np.linalg.norm(b) <= 1e-8
    # dense solve itself: (K + mu I) a = b by a library solve
    K = oracle.kernel_matrix(X, X, G, 0.1) + 1e-4 * np.eye(400)
    assert np.allclose(a, np.linalg.solve(K, b), rtol=1e-8, atol=1e-8)


def test_pcg_exact_preconditioner_one_iteration():
    X = pts(60, 2, 29)
    b = inputs.rhs(60, 1, 30)[:, 0]
    fn = oracle.afn_build(X, G, 0.3, 1e-2, 60, 4)           # k = n  =>  M = K + mu I
    x, it, rel, st = oracle.pcg(fn, b, 1e-10)
    assert st == 0 and it == 1
    fw = oracle.afn_build(X, G, 0.3, 1e-2, 10, 50)          # full FSAI pattern
    x, it, rel, st = oracle.pcg(fw, b, 1e-10)
    assert st == 0 and it == 1


def test_cg_two_eigenvalues_two_iterations():
    # identical points: K = 11^T, K + mu I has 2 distinct eigenvalues -> CG in 2 steps
    X = np.zeros((30, 3))
    b = inputs.rhs(30, 1, 31)[:, 0]
    f = oracle.afn_build(X, G, 1.0, 0.5, 0, 1)
    x, it, rel, st = oracle.pcg(f, b, 1e-12, identity=True)
    assert st == 0 and it == 2
    A = np.ones((30, 30)) + 0.5 * np.eye(30)
    assert np.allclose(x, np.linalg.solve(A, b), rtol=1e-10)


def test_pcg_afn_beats_cg_and_multi_rhs():
    X = pts(500, 3, 32)
    B = inputs.rhs(500, 2, 33)
    f = oracle.afn_build(X, G, 0.15, 1e-4, 60, 12)
    x, it, rel, st = oracle.pcg(f, B, 1e-6)
    _, itcg, _, _ = oracle.pcg(f, B, 1e-6, identity=True, max_iter=2000)
    assert np.all(st == 0) and np.all(rel <= 1e-6)
    assert np.all(it < itcg)
    assert np.all(oracle.true_relres(X, G, 0.15, 1e-4, x, B) <= 1e-6)


def test_true_relres_special_values():
    # x = 0 leaves r = b (relative residual exactly 1); the dense solve leaves rounding only;
    # a zero column b has the solution 0 (value 0) and any other x is wrong (value inf)
    X = pts(40, 2, 35)
    A = np.exp(-((X[:, None, :] - X[None, :, :]) ** 2).sum(-1) / 0.3 ** 2) + 1e-2 * np.eye(40)
    B = inputs.rhs(40, 3, 36)
    B[:, 2] = 0.0
    x = np.linalg.solve(A, B)
    rel = oracle.true_relres(X, G, 0.3, 1e-2, x, B)
    assert np.all(rel[:2] < 1e-12) and rel[2] == 0.0
    rel0 = oracle.true_relres(X, G, 0.3, 1e-2, np.zeros_like(B), B)
    assert np.array_equal(rel0, np.array([1.0, 1.0, 0.0]))
    x[0, 2] = 1e-3
    assert oracle.true_relres(X, G, 0.3, 1e-2, x, B)[2] == np.inf


# -------------------------------------------------------- eigen / Alg. 4 ---
def test_tridiagonalize_and_sturm_against_eigvalsh():
    X = pts(80, 3, 34)
    A = oracle.kernel_matrix(X, X, M32, 0.3)
    ev = np.linalg.eigvalsh(A)
    dg, of = oracle.tridiagonalize(A)
    for s in (1e-6, 1e-3, 0.1, 1.0, 5.0):
        assert oracle.sturm_count(dg, of, s) == int((ev < s).sum())
    assert oracle.tridiag_max_eig(dg, of) == pytest.approx(ev.max(), rel=1e-12)
    T = np.diag(dg) + np.diag(of, 1) + np.diag(of, -1)
    assert np.allclose(np.linalg.eigvalsh(T), ev, atol=1e-12)


def _rank_estimate_library(X, ker, l, mu, m, seed, k_max):
    """Alg. 4 by linear scan with numpy eigvalsh and numpy Schur complements."""
    n, d = X.shape
    m = min(m, n)
    sub = oracle.uniform_sample(n, m, seed)
    Xs = X[sub] * (m / n) ** (1.0 / d)
    o = oracle.fps(Xs, m, 0)
    Ko = oracle.kernel_matrix(Xs[o], Xs[o], ker, l)
    lmax = np.linalg.eigvalsh(Ko).max()
    r = m
    for rr in range(1, m):
        A, B, Cc = Ko[:rr, :rr], Ko[:rr, rr:], Ko[rr:, rr:]
        E = Cc - B.T @ np.linalg.solve(A, B)
        if np.linalg.eigvalsh(E).max() < 0.1 * lmax:
            r = rr
            break
    if r * n >= 2000 * m:
        k = -(-r * n // m)
    else:
        Ku = oracle.kernel_matrix(X[sub], X[sub], ker, l)
        k = int((np.linalg.eigvalsh(Ku) > 0.1 * mu).sum())
    return max(1, min(k, k_max, n)), r


@pytest.mark.parametrize("l,n", [(0.05, 3000), (0.3, 3000), (1.0, 3000), (3.0, 800)])
def test_rank_estimate_matches_library_scan(l, n):
    X = pts(n, 3, 35)
    k, r, br = oracle.rank_estimate(X, G, l, 1e-2, m=120, seed=7, k_max=100000)
    k2, r2 = _rank_estimate_library(X, G, l, 1e-2, 120, 7, 100000)
    assert (k, r) == (k2, r2)
    assert br == (0 if r * n >= 2000 * 120 else 1)


def test_rank_estimate_extremes():
    X = pts(4000, 3, 36)
    # l tiny: K ~ I, the Nystrom error stays 1 until r = m -> k = n
    k, r, br = oracle.rank_estimate(X, G, 1e-4, 1e-2, m=100, seed=1, k_max=10**6)
    assert r == 100 and k == 4000 and br == 0
    # l huge: K ~ 11^T, rank 1 -> eigenvalue branch, a handful of eigenvalues above 0.1 mu
    k, r, br = oracle.rank_estimate(X, G, 1e4, 1e-2, m=100, seed=1, k_max=10**6)
    assert r == 1 and br == 1 and 1 <= k <= 3
    # cap
    k, r, br = oracle.rank_estimate(X, G, 1e-4, 1e-2, m=100, seed=1, k_max=500)
    assert k == 500


# ----------------------------------------------- Nystrom branch (Alg. 5) ---
def test_jacobi_eig_against_eigvalsh():
    A = inputs.rng(41).standard_normal((30, 30))
    A = A + A.T
    w, V = oracle.jacobi_eig(A)
    assert np.allclose(V.T @ V, np.eye(30), atol=1e-13)
    assert np.allclose(A @ V, V * w, atol=1e-11)
    assert np.allclose(np.sort(w), np.linalg.eigvalsh(A), atol=1e-11)


def _nys_dense(f):
    # K_nys = Y (K_SS + nu I)^{-1} Y^T written out with library solves
    Xp, k = f["Xp"], f["k"]
    n = Xp.shape[0]
    Y = oracle.kernel_matrix(Xp, Xp[:k], f["kernel"], f["l"])
    Kss = Y[:k] + n * 2.0 ** -52 * np.eye(k)
    return Y @ np.linalg.solve(Kss, Y.T)


@pytest.mark.parametrize("ker,l,k", [(G, 0.3, 40), (M32, 0.5, 25)])
def test_nystrom_factors_closed_form(ker, l, k):
    X = pts(200, 3, 43)
    f = oracle.nystrom_build(X, ker, l, 1e-2, k)
    U, lam, r = f["U"][:, :f["r"]], f["lam"][:f["r"]], f["r"]
    assert r == k                                    # FPS landmarks: K_SS well conditioned
    assert np.allclose(U.T @ U, np.eye(r), atol=1e-10)
    Kn = _nys_dense(f)
    assert np.abs(U @ np.diag(lam) @ U.T - Kn).max() <= 1e-9 * np.abs(Kn).max()
    # the landmark rows are reproduced: K_nys[S, :] = K[S, :] (up to the shift)
    K = oracle.kernel_matrix(f["Xp"], f["Xp"], ker, l)
    assert np.abs(Kn[:k] - K[:k]).max() <= 1e-8


@pytest.mark.parametrize("mu", [1e-1, 1e-3])
def test_nystrom_apply_inverts_M(mu):
    # eq. (nystrom1-smw) against the direct inverse of K_nys + mu I
    X = pts(150, 2, 44)
    f = oracle.nystrom_build(X, G, 0.25, mu, 30)
    Kn = _nys_dense(f)
    r = inputs.rhs(150, 1, 45)[:, 0]
    s = oracle.nystrom_apply(f, r)
    ref = np.linalg.solve(Kn + mu * np.eye(150), r)
    assert np.abs(s - ref).max() <= 1e-8 * np.abs(ref).max()


def test_nystrom_all_landmarks_one_step():
    # k = n: K_nys = K (up to the shift), so M = K + mu I and PCG needs one product
    X = pts(60, 3, 46)
    f = oracle.nystrom_build(X, G, 0.15, 1e-2, 60)
    b = inputs.rhs(60, 1, 47)[:, 0]
    x, it, rel, st = oracle.pcg_nystrom(f, b, 1e-10)
    assert st == 0 and it <= 2 and rel <= 1e-10


def test_pcg_nystrom_reaches_dense_solution():
    X = pts(400, 3, 48)
    f = oracle.nystrom_build(X, M32, 0.4, 1e-2, 60)
    b = inputs.rhs(400, 1, 49)[:, 0]
    x, it, rel, st = oracle.pcg_nystrom(f, b, 1e-10, max_iter=400)
    xd = oracle.dense_solve(X, M32, 0.4, 1e-2, b)
    assert st == 0 and rel <= 1e-10
    assert np.abs(x - xd).max() <= 1e-8 * np.abs(xd).max()
    # and it is a better preconditioner than none
    fa = oracle.afn_build(X, M32, 0.4, 1e-2, 0, 1)
    _, it_cg, _, _ = oracle.pcg(fa, b, 1e-10, max_iter=400, identity=True)
    assert it < it_cg


def test_strategy_threshold_selects_branch():
    X = pts(300, 3, 50)
    k = oracle.rank_estimate(X, G, 0.3, 1e-2, m=100, seed=3, k_max=300)[0]
    assert 0 < k < 300
    below = oracle.strategy(X, G, 0.3, 1e-2, 300, 16, m=100, seed=3, threshold=k + 1)
    above = oracle.strategy(X, G, 0.3, 1e-2, 300, 16, m=100, seed=3, threshold=k)
    assert below["precond"] == "nystrom" and below["k"] == k
    assert above["precond"] == "afn" and above["k"] == k
