"""Host replay of the FP32 pre-test that keeps the FSAI pattern search exact.

Once a row's candidate list is full, the KNN kernel skips a point j when its
FP32 squared distance z exceeds a cut computed from the worst candidate's
FP64 distance wv:

    cut(wv) = (wv + delta (2 sqrt(d wv) + d delta)) / (1 - (d + 2) 2^-24),
    delta = 2^-22 M (1 + 2^-20),  M = max |coordinate|,

every operation rounded upward in FP32.  The pattern stays exactly that of an
FP64 scan only if a point with r2 <= wv always has z <= cut(wv); since the
cut grows with wv, it is enough that z <= cut(r2) for every pair.  This file
replays the kernel's arithmetic (FP32 coordinates, FP32 differences, squares
and running sum rounded to nearest, no fused multiply-add; the cut with
upward rounding) on point sets built to stress it, and checks that inequality
for every pair, that the cut is not loose by more than the analysis allows,
and that a cut without its error terms would be violated.  On these sets z
gets at most 0.36 of the way from r2 to the cut.
"""

import numpy as np
import pytest

from paper_2304_05460_gb300 import inputs

f32, f64 = np.float32, np.float64


def _ru(x64):
    """Round FP64 values up to FP32."""
    y = np.asarray(x64, dtype=f64).astype(f32)
    low = y.astype(f64) < x64
    y[low] = np.nextafter(y[low], f32(np.inf))
    return y


def _rd(x):
    y = f32(x)
    return np.nextafter(y, f32(-np.inf)) if f64(y) > x else y


def cut(wv64, d, M, terms=True):
    """The kernel's cut, each operation rounded upward in FP32."""
    dlt = _ru(np.array([M * 2.0 ** -22 * (1.0 + 2.0 ** -20)]))[0]
    den = _rd(1.0 - (d + 2) * 2.0 ** -24)
    fd = f32(d)
    ddl = _ru(f64(fd) * f64(dlt))
    wv = _ru(wv64)
    if not terms:
        return wv
    sq = _ru(np.sqrt(_ru(f64(fd) * wv.astype(f64)).astype(f64)))
    b = _ru(f64(dlt) * _ru(_ru(2.0 * sq.astype(f64)).astype(f64) + f64(ddl)).astype(f64))
    return _ru(_ru(wv.astype(f64) + b.astype(f64)).astype(f64) / f64(den))


def z32(xi, X):
    """FP32 squared distances of row point xi to the rows of X, as the kernel sums them."""
    xif = xi.astype(f32)
    Xf = X.astype(f32)
    z = np.zeros(X.shape[0], f32)
    for t in range(X.shape[1]):
        u = (xif[t] - Xf[:, t]).astype(f32)
        z = (z + (u * u).astype(f32)).astype(f32)
    return z


def r2_64(xi, X):
    r = np.zeros(X.shape[0])
    for t in range(X.shape[1]):
        u = xi[t] - X[:, t]
        r = r + u * u
    return r


def _point_sets():
    g = inputs.rng(81)
    sets = []
    for d in (1, 2, 3, 8, 16):
        sets.append(("normal", d, g.standard_normal((400, d))))
        # far from the origin, tiny spread: coordinate rounding dominates the differences
        sets.append(("offset", d, 1000.0 + 1e-3 * g.standard_normal((400, d))))
        # coordinates near the extremes +-M with duplicates and near-duplicates
        base = g.uniform(-1.0, 1.0, (200, d)) * 3.7e5
        near = base + g.standard_normal((200, d)) * 1e-2
        sets.append(("extreme", d, np.concatenate([base, near, base[:20]])))
        sets.append(("tiny", d, 1e-30 * g.standard_normal((400, d))))
    return sets


@pytest.mark.parametrize("kind,d,X", _point_sets(), ids=lambda v: v if isinstance(v, (str, int)) else "")


def test_fp32_distance_never_exceeds_the_cut(kind, d, X):
    M = float(np.abs(X).max())
    for i in range(0, X.shape[0], 7):
        z = z32(X[i], X)
        r2 = r2_64(X[i], X)
        assert np.all(z <= cut(r2, d, M)), (kind, d, i)


def test_cut_is_not_loose():
    # the cut is the analysis's bound, (1 + (d + 2) 2^-24) wv plus the delta terms, up to
    # a few FP32 units in the last place of its upward-rounded steps
    d = 8
    X = inputs.normal_points(300, d, 82)
    M = float(np.abs(X).max())
    r2 = r2_64(X[0], X)[1:]
    c = cut(r2, d, M).astype(f64)
    dl = M * 2.0 ** -22
    ulp = np.spacing(r2.astype(f32)).astype(f64)
    allowed = r2 * (1 + (d + 2) * 2.0 ** -24) + dl * (2 * np.sqrt(d * r2) + d * dl) * 1.01 + 4 * ulp
    assert np.all(c <= allowed)
    assert np.all(c >= r2 + dl * 2 * np.sqrt(d * r2))


def test_cut_without_its_error_terms_is_violated():
    # the same replay with the cut reduced to wv itself: some pair's FP32 distance
    # lies above its FP64 distance, so the error terms are needed
    g = inputs.rng(83)
    X = 1000.0 + 1e-3 * g.standard_normal((400, 3))
    M = float(np.abs(X).max())
    bad = 0
    for i in range(0, 400, 7):
        bad += int(np.sum(z32(X[i], X) > cut(r2_64(X[i], X), 3, M, terms=False)))
    assert bad > 0
