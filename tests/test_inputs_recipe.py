"""The seeded workload generators against the recipe they state.

Each workload's shapes, parameters and value distributions are checked here:
exact properties (shapes, layouts, ranges, parameter values, determinism) and
statistical ones with bounds of several standard errors, so that a wrong
distribution, scale or parameter fails while a reseed would not.
"""
import math

import numpy as np
import pytest

from paper_2304_05460_gb300 import inputs as I


def test_rng_is_pcg64_and_deterministic():
    a = I.rng(7).standard_normal(16)
    b = np.random.Generator(np.random.PCG64(7)).standard_normal(16)
    assert np.array_equal(a, b)
    assert not np.array_equal(a, I.rng(8).standard_normal(16))
    assert I.rhs(100, 3, 5).flags.f_contiguous
    assert I.rhs(100, 3, 5).shape == (100, 3)


def test_uniform_cube_3d():
    s = I.uniform_cube_3d()
    assert s.X.shape == (2000, 3) and s.X.dtype == np.float64
    assert s.X.min() >= 0.0 and s.X.max() < 1.0
    assert s.B.shape == (2000, 1) and s.B.flags.f_contiguous
    assert (s.kernel, s.l, s.mu, s.k, s.w) == (I.GAUSSIAN, 0.1, 1e-4, 200, 32)
    assert s.rank_mode == "fixed" and s.landmarks == "fps" and s.fps_start == 0
    # U[0,1]: mean 1/2, variance 1/12 per coordinate (6000 samples)
    assert abs(s.X.mean() - 0.5) < 5 * math.sqrt(1 / 12 / s.X.size)
    assert abs(s.X.var() - 1 / 12) < 0.005


def test_normal_8d():
    s = I.normal_8d()
    assert s.X.shape == (50_000, 8) and s.B.shape == (50_000, 32)
    assert s.B.flags.f_contiguous
    assert (s.kernel, s.l, s.mu, s.k, s.w) == (I.GAUSSIAN, 1.0, 1e-2, 4000, 64)
    assert s.rank_mode == "estimate"
    # N(0, I_8): per-coordinate mean 0 and unit variance, coordinates uncorrelated
    se = 1.0 / math.sqrt(s.n)
    assert np.all(np.abs(s.X.mean(0)) < 5 * se)
    assert np.all(np.abs(s.X.var(0) - 1.0) < 5 * math.sqrt(2.0) * se)
    C = np.corrcoef(s.X.T)
    assert np.all(np.abs(C - np.eye(8)) < 5 * se)
    # the length scale only changes l; the one-RHS form is the first column of the 32
    s2 = I.normal_8d(l=2.0, nrhs=1)
    assert s2.l == 2.0 and np.array_equal(s2.X, s.X)
    assert s2.B.shape == (50_000, 1) and np.array_equal(s2.B[:, 0], s.B[:, 0])


def test_clusters_3d():
    s = I.clusters_3d()
    n = 200_000
    assert s.X.shape == (n, 3) and s.B.shape == (n, 64)
    assert (s.kernel, s.l, s.mu, s.k, s.w) == (I.MATERN32, 0.05, 1e-3, 2000, 50)
    # the centres are the generator's first draw
    centres = I.rng(1003).uniform(0.0, 1.0, size=(3, 3))
    d2 = ((s.X[:, None, :] - centres[None, :, :]) ** 2).sum(-1)
    near = d2.min(1)
    sigma = 0.1
    # a clustered point lies within sigma of its centre with probability
    # P(chi2_3 <= 1) = erf(1/sqrt 2) - sqrt(2/pi) e^(-1/2); a uniform one with
    # probability at most 3 * (4/3) pi sigma^3 (balls clipped by the cube give less)
    p_in = math.erf(1 / math.sqrt(2)) - math.sqrt(2 / math.pi) * math.exp(-0.5)
    lo = 0.8 * n * p_in
    hi = lo + 0.2 * n * 3 * (4 / 3) * math.pi * sigma ** 3
    cnt = int((near <= sigma ** 2).sum())
    sd = math.sqrt(0.8 * n * p_in * (1 - p_in))
    assert lo - 5 * sd <= cnt <= hi + 5 * sd
    # equal cluster weights: each centre holds about a third of the near points
    which = d2.argmin(1)[near <= sigma ** 2]
    share = np.bincount(which, minlength=3) / len(which)
    assert np.all(np.abs(share - 1 / 3) < 0.03)
    # the remaining 20 % are uniform: no point outside the cube is far from a centre,
    # and the order is shuffled (both halves hold the same share of near points)
    out = np.any((s.X < 0.0) | (s.X > 1.0), axis=1)
    assert out.any() and np.all(near[out] < (8 * sigma) ** 2)
    h = n // 2
    f1 = (near[:h] <= sigma ** 2).mean()
    f2 = (near[h:] <= sigma ** 2).mean()
    assert abs(f1 - f2) < 0.01


def test_paper_cube_3d():
    for n in (1000, 160_000):
        s = I.paper_cube_3d(n=n)
        edge = n ** (1.0 / 3.0)
        assert s.X.shape == (n, 3) and s.B.shape == (n, 1)
        assert s.X.min() >= 0.0 and s.X.max() < edge
        assert s.X.max() > 0.99 * edge and s.X.min() < 0.01 * edge
        assert s.B.min() >= -0.5 and s.B.max() < 0.5
        assert abs(s.B.mean()) < 5 * math.sqrt(1 / 12 / n)
        assert (s.kernel, s.mu, s.w) == (I.GAUSSIAN, 1e-4, 100)
        assert s.rank_mode == "estimate"
    # unit density: about one point per unit volume in every octant
    s = I.paper_cube_3d()
    oct_ = (s.X >= 0.5 * 160_000 ** (1 / 3)).astype(int) @ np.array([1, 2, 4])
    cnt = np.bincount(oct_, minlength=8)
    assert np.all(np.abs(cnt - 20_000) < 5 * math.sqrt(20_000))
    assert len(I.PAPER_GAUSSIAN_L2) == len(I.PAPER_MATERN_INV_L) == 11


def test_median_pairwise_distance_exact_and_estimated():
    X = I.normal_points(301, 4, 11)
    D = np.sqrt(((X[:, None, :] - X[None, :, :]) ** 2).sum(-1))
    v = np.sort(D[np.triu_indices(301, 1)])
    assert I.median_pairwise_distance(X, 0) == pytest.approx(v[(len(v) - 1) // 2], rel=1e-12)
    # above the exact limit: 10^5 sampled pairs estimate the median within a few 0.1 %
    pdist = pytest.importorskip("scipy.spatial.distance").pdist
    Y = I.normal_points(3000, 8, 12)
    exact = np.median(pdist(Y))
    assert I.median_pairwise_distance(Y, 5) == pytest.approx(exact, rel=0.01)


def test_batched_512_prefix():
    systems = I.batched_512(count=48)
    assert len(systems) == 48
    for s in systems:
        assert 256 <= s.n < 8192 and 2 <= s.d <= 16
        assert s.B.shape == (s.n, 8) and s.B.flags.f_contiguous
        assert s.kernel == I.GAUSSIAN and s.w == 32 and s.k == min(s.n // 4, 1000)
        assert 1e-4 <= s.mu <= 1e-1 and s.landmarks == "auto"
        med = I.median_pairwise_distance(s.X, s.seed + 7)
        assert 0.1 * med <= s.l <= 10.0 * med
        assert abs(s.X.mean()) < 6 / math.sqrt(s.X.size)
    assert len({s.seed for s in systems}) == 48
    # log-uniform n: ln n spread over [ln 256, ln 8192] (mean within 4 standard errors)
    ln = np.log([s.n for s in systems])
    mid, half = 0.5 * (math.log(256) + math.log(8192)), 0.5 * math.log(32)
    assert abs(ln.mean() - mid) < 4 * half / math.sqrt(3 * len(ln))
    # the same seed gives the same systems
    again = I.batched_512(count=2)
    assert np.array_equal(again[1].X, systems[1].X) and again[1].l == systems[1].l


def test_serving_stream():
    reqs = I.serving_stream()
    assert len(reqs) == 10_000 and [r["id"] for r in reqs] == list(range(10_000))
    t = np.array([r["t"] for r in reqs])
    assert np.all(np.diff(t) > 0) and t[0] > 0
    # Poisson arrivals at rate 1/s: exponential gaps of mean 1 and variance 1
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert abs(gaps.mean() - 1.0) < 5 / math.sqrt(len(gaps))
    assert abs(gaps.var() - 1.0) < 0.1
    assert abs(I.serving_stream(count=2000, rate=4.0)[-1]["t"] / 2000 - 0.25) < 0.03
    n = np.array([r["n"] for r in reqs])
    assert n.min() >= 1000 and n.max() < 100_000
    assert abs(np.log(n).mean() - 0.5 * math.log(1e8)) < 0.05
    assert {r["d"] for r in reqs} == {3, 8, 16}
    assert abs(np.mean([r["kernel"] for r in reqs]) - 0.5) < 0.03
    nr = [r["nrhs"] for r in reqs]
    assert min(nr) == 1 and max(nr) == 16
    assert all(0.1 <= r["lfac"] <= 10 and 1e-4 <= r["mu"] <= 1e-1 for r in reqs)
    assert len({r["seed"] for r in reqs}) == 10_000
    s = I.serving_system(reqs[3])
    r = reqs[3]
    assert s.X.shape == (r["n"], r["d"]) and s.B.shape == (r["n"], r["nrhs"])
    assert s.kernel == r["kernel"] and s.mu == r["mu"] and s.k == min(r["n"] // 4, 1000)
    assert s.l == pytest.approx(I.median_pairwise_distance(s.X, r["seed"] + 7) * r["lfac"])
