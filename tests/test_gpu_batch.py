"""GPU parity of the batched (grouped) solve against the FP64 oracle.

Bars (as for single systems): every column's final relative residual
||b - (K + mu I) x|| / ||b||, recomputed by the oracle in FP64, is <= tol;
the factors of each system are the single-system build's (k, w); a system's
solution is bit-identical alone and in a mix of other systems (the grouped
kernels never combine work of two systems); iteration counts stay within a
band of the single-system mixed solve of the same system (the two replace the
FP64 residual at slightly different iterations).
"""
import math

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


def system(n, d, ker, lfac, mu, nrhs, seed, k=None, w=32):
    g = inputs.rng(seed)
    X = g.standard_normal((n, d))
    B = np.asfortranarray(g.standard_normal((nrhs, n)).T)
    l = inputs.median_pairwise_distance(X, seed + 7) * lfac
    return dict(points=X, kernel=ker, l=l, mu=mu, k_max=min(n // 4, 1000) if k is None else k,
                fsai_nnz=w), B


# uneven sizes, dimensions, kernels, scales and widths (1 .. 16 columns,
# ragged column groups), plus the degenerate k = 0 and k = n systems
MIX = [(300, 2, G, 0.5, 1e-1, 1, 11), (517, 3, M32, 1.0, 1e-2, 3, 12),
       (1000, 5, G, 2.0, 1e-3, 8, 13), (1500, 9, M32, 0.7, 1e-2, 9, 14),
       (2300, 12, G, 1.3, 3e-3, 16, 15), (777, 16, M32, 3.0, 1e-2, 5, 16),
       (400, 4, G, 1.0, 1e-2, 2, 17, 0), (260, 3, M32, 0.8, 1e-2, 4, 18, 260)]


def make_mix():
    out = []
    for m in MIX:
        sy, B = system(*m[:7], k=m[7] if len(m) > 7 else None)
        out.append((sy, B))
    return out


def check_residuals(sy, x, B, tol):
    X = sy["points"]
    x2 = x.reshape(X.shape[0], -1)
    rel = oracle.true_relres(X, sy["kernel"], sy["l"], sy["mu"], x2, B)
    rel = np.where(np.linalg.norm(B, axis=0) > 0, rel, 0.0)
    assert np.max(rel) <= tol, rel
    return rel


def test_batched_mix_reaches_tol(afn):
    mix = make_mix()
    tol = 1e-6
    b = afn.afn_build_batched([m[0] for m in mix], seed=5, max_iter=2000)
    xs, info = afn.afn_solve_batched(b, [m[1] for m in mix], tol)
    assert info["status"] == afn.AFN_OK, info
    assert info["converged"] == info["columns"] == sum(m[1].shape[1] for m in mix)
    for s, (sy, B) in enumerate(mix):
        bi = afn.afn_batch_build_info(b, s)
        n = sy["points"].shape[0]
        assert bi.k == min(sy["k_max"], n) and bi.w == min(32, max(n - bi.k, 1))
        check_residuals(sy, np.asarray(xs[s]), B, tol)


def test_batched_matches_single_mixed(afn):
    mix = make_mix()[:6]
    tol = 1e-6
    b = afn.afn_build_batched([m[0] for m in mix], seed=5, max_iter=2000,
                              precision=afn.PREC_MIXED)
    xs, info = afn.afn_solve_batched(b, [m[1] for m in mix], tol)
    for s, (sy, B) in enumerate(mix):
        # the grouped solves run the W products on the CUDA cores in FP32: the single
        # solve takes the same apply (apply_tc = 0) for a like-for-like comparison
        h = afn.afn_build(sy["points"], sy["kernel"], sy["l"], sy["mu"], sy["k_max"],
                          sy["fsai_nnz"], precision=afn.PREC_MIXED, seed=5, max_iter=2000,
                          apply_tc=0)
        x1, i1 = afn.afn_solve(h, B, tol)
        it_b, it_1 = info["iters"][s], i1["iters"]
        # the grouped apply sums in 8-column groups, the single one in its own pieces: the
        # rounding differs, so the mixed iteration counts agree only within a band
        assert np.all(np.abs(it_b - it_1) <= np.maximum(6, 0.25 * it_1)), (s, it_b, it_1)
        # ||x - a*|| <= ||A^{-1}||_2 ||b - A x|| <= tol ||b|| / lambda_min(A)
        X = sy["points"]
        if X.shape[0] <= 1500:
            A = oracle.kernel_matrix(X, X, sy["kernel"], sy["l"]) + sy["mu"] * np.eye(X.shape[0])
            lmin = np.linalg.eigvalsh(A)[0]
            a = oracle.dense_solve(X, sy["kernel"], sy["l"], sy["mu"], B[:, 0])
            err = np.linalg.norm(np.asarray(xs[s]).reshape(X.shape[0], -1)[:, 0] - a)
            assert err <= 1.01 * tol * np.linalg.norm(B[:, 0]) / lmin
        afn.afn_free(h)


def test_alone_and_in_mix_bit_identical(afn):
    mix = make_mix()
    tol = 1e-6
    b_all = afn.afn_build_batched([m[0] for m in mix], seed=5, max_iter=2000)
    xs, _ = afn.afn_solve_batched(b_all, [m[1] for m in mix], tol)
    for s in (1, 4, 7):
        b1 = afn.afn_build_batched([mix[s][0]], seed=5, max_iter=2000)
        x1, _ = afn.afn_solve_batched(b1, [mix[s][1]], tol)
        assert np.array_equal(np.asarray(x1[0]), np.asarray(xs[s])), s


def test_batched_zero_column_and_device_memory(afn):
    torch = pytest.importorskip("torch")
    sy, B = system(900, 3, G, 1.0, 1e-2, 4, 31)
    B[:, 2] = 0.0
    sy2, B2 = system(350, 6, M32, 0.5, 1e-3, 1, 32)
    for s_ in (sy, sy2):
        s_["points"] = torch.tensor(s_["points"], device="cuda")
    b = afn.afn_build_batched([sy, sy2], seed=1)
    xs, info = afn.afn_solve_batched(b, [torch.tensor(B, device="cuda"),
                                         torch.tensor(B2, device="cuda")], 1e-6)
    assert info["status"] == afn.AFN_OK
    assert xs[0].is_cuda
    x0 = xs[0].cpu().numpy()
    assert np.all(x0[:, 2] == 0.0)
    sy["points"] = sy["points"].cpu().numpy()
    check_residuals(sy, x0, B, 1e-6)


def test_batched_rejects_bad_input(afn):
    sy, B = system(300, 3, G, 1.0, 1e-2, 2, 41)
    with pytest.raises(afn.AfnError) as e:
        afn.afn_build_batched([sy], precision=7)
    assert e.value.status == afn.AFN_ERR_ARG
    bad = dict(sy, mu=-1.0)
    with pytest.raises(afn.AfnError) as e:
        afn.afn_build_batched([sy, bad])
    assert e.value.status == afn.AFN_ERR_ARG and "system 1" in str(e.value)
    b = afn.afn_build_batched([sy])
    Bn = B.copy()
    Bn[3, 1] = np.nan
    with pytest.raises(afn.AfnError) as e:
        afn.afn_solve_batched(b, [Bn], 1e-6)
    assert e.value.status == afn.AFN_ERR_ARG


def test_batched_512_workload_sample(afn):
    """Sixteen systems of the 512-system batched workload (n log-uniform in
    [256, 8192], d in 2..16, l = median distance x log-uniform [0.1, 10], mu
    log-uniform [1e-4, 1e-1], k = min(n/4, 1000), w = 32, 8 RHS) solved
    together; residuals checked by the oracle on the systems with n <= 3000."""
    systems = inputs.batched_512()[:16]
    tol = 1e-6
    sys_args = [dict(points=s.X, kernel=s.kernel, l=s.l, mu=s.mu, k_max=s.k, fsai_nnz=s.w)
                for s in systems]
    b = afn.afn_build_batched(sys_args, seed=1004, max_iter=3000)
    xs, info = afn.afn_solve_batched(b, [s.B for s in systems], tol)
    assert info["converged"] == info["columns"], (info["converged"], info["columns"])
    for s, sy in enumerate(sys_args):
        if sy["points"].shape[0] <= 3000:
            check_residuals(sy, np.asarray(xs[s]), systems[s].B, tol)


def test_auto_precision_routes_small_mu(afn):
    """AFN_PREC_AUTO sends a system whose FP32 matvec error would swamp mu
    (mu = 1e-4, length-scale 4x the median distance) to the DF path (FP64 PCG,
    double-float matvec) and keeps the easy ones mixed; both reach tol in one
    batched call, and the DF system needs few iterations."""
    hard, Bh = system(2500, 8, G, 4.0, 1e-4, 8, 51)
    easy, Be = system(1200, 5, M32, 0.7, 1e-2, 8, 52)
    b = afn.afn_build_batched([hard, easy], seed=5, max_iter=2000)
    ih, ie = afn.afn_batch_build_info(b, 0), afn.afn_batch_build_info(b, 1)
    assert ih.precision == afn.PREC_DF and ih.rho32 > 0.3
    assert ie.precision == afn.PREC_MIXED and 0 < ie.rho32 <= 0.3
    xs, info = afn.afn_solve_batched(b, [Bh, Be], 1e-6)
    assert info["status"] == afn.AFN_OK
    check_residuals(hard, np.asarray(xs[0]), Bh, 1e-6)
    check_residuals(easy, np.asarray(xs[1]), Be, 1e-6)
    assert info["iters"][0].max() < 200
