"""Pins for the oracle's sampled-output functions (no GPU).

The full-size parity tests compare the CUDA path with the oracle on a sample
of rows: ``matvec_rows`` (rows of (K + mu I) p, eq. (Problem)), ``fsai_rows``
(rows of G, Alg. 1 on the Schur complement) and ``knn_rows`` (rows of the
FSAI pattern, Sec. 3.1).  Each must reproduce, exactly, the same rows of the
oracle's full computation (``matvec``, ``afn_build``'s G and ``knn_pattern``),
which are themselves pinned to closed forms and brute force in
test_oracle_pins.py.  The sums run in the same order on both sides, so the
comparison is bitwise.  Row sets are ragged (first, last, repeated and
unsorted rows), both kernels and several right-hand sides are covered, so a
wrong output index, a transposed K12 column or a shifted pattern row fails.
"""
import numpy as np
import pytest

import oracle
from paper_2304_05460_gb300 import inputs

G, M32 = oracle.GAUSSIAN, oracle.MATERN32


def _rows(n, seed, count):
    r = inputs.rng(seed).choice(n, size=min(count, n), replace=False)
    return np.concatenate([[n - 1, 0], r, [n - 1, 3 % n]]).astype(np.int64)


@pytest.mark.parametrize("ker,n,d,nrhs", [(G, 97, 3, 1), (M32, 130, 5, 4), (G, 61, 8, 33)])
def test_matvec_rows_equals_full_product_rows(ker, n, d, nrhs):
    X = inputs.normal_points(n, d, 40 + n)
    P = inputs.rhs(n, nrhs, 41 + n)
    l, mu = 0.8 * np.sqrt(d), 3e-3
    rows = _rows(n, 42 + n, 17)
    full = oracle.matvec(X, ker, l, mu, P).reshape(n, nrhs)
    got = oracle.matvec_rows(X, ker, l, mu, P, rows)
    assert got.shape == (len(rows), nrhs)
    assert np.array_equal(got, full[rows])
    # 1-D p gives one column
    got1 = oracle.matvec_rows(X, ker, l, mu, P[:, 0], rows)
    assert np.array_equal(got1[:, 0], full[rows, 0])


@pytest.mark.parametrize("ker,n,k,w", [(G, 140, 23, 9), (M32, 120, 40, 17), (G, 90, 0, 6),
                                       (M32, 75, 30, 1)])
def test_fsai_rows_equals_build_rows(ker, n, k, w):
    X = inputs.uniform_points(n, 3, 50 + n)
    l, mu = 0.3, 1e-3
    f = oracle.afn_build(X, ker, l, mu, k, w)
    nr = f["nr"]
    rows = _rows(nr, 51 + n, 11)
    got = oracle.fsai_rows(f["Xp"], ker, l, mu, f["k"], f["w"], f["L"], f["pattern"], rows)
    assert got.shape == (len(rows), f["w"])
    assert np.array_equal(got, f["G"][rows])


@pytest.mark.parametrize("nr,d,w", [(150, 3, 1), (150, 2, 5), (220, 8, 33), (64, 3, 64)])
def test_knn_rows_equals_pattern_rows(nr, d, w):
    X = inputs.uniform_points(nr, d, 60 + nr)
    pat, _ = oracle.knn_pattern(X, w)
    rows = _rows(nr, 61 + nr, 19)
    got = oracle.knn_rows(X, w, rows)
    assert got.shape == (len(rows), w)
    assert np.array_equal(got, pat[rows])


def test_knn_rows_rejects_out_of_range():
    X = inputs.uniform_points(10, 2, 1)
    with pytest.raises(ValueError):
        oracle.knn_rows(X, 3, [10])


def test_fsai_rows_rejects_out_of_range():
    X = inputs.uniform_points(12, 2, 2)
    L = np.eye(4)
    pat = np.full((8, 3), -1, np.int32)
    pat[:, 0] = np.arange(8)
    for rows, k in (([8], 4), ([-1], 4), ([0], 13)):
        with pytest.raises(ValueError):
            oracle.fsai_rows(X, oracle.GAUSSIAN, 0.5, 1e-2, k, 3, L, pat, rows)


def test_matvec_rows_rejects_out_of_range():
    X = inputs.uniform_points(10, 2, 3)
    for rows in ([10], [-1]):
        with pytest.raises(ValueError):
            oracle.matvec_rows(X, oracle.GAUSSIAN, 0.5, 1e-2, np.ones(10), rows)
