"""Seeded synthetic inputs for the AFN-PCG workloads.

This module holds none of the method's arithmetic: it only draws points,
right-hand sides and per-system parameters with numpy's PCG64 generator.
Both the CUDA path and the CPU oracle take their inputs from here.

Workloads (points drawn first, then right-hand sides; seed 1000 + c):

* ``uniform_cube_3d``  n=2000, U[0,1]^3, Gaussian l=0.1, mu=1e-4, k=200 FPS
  landmarks from index 0, w=32, one N(0,1) right-hand side.
* ``normal_8d``        n=50000, N(0, I_8), Gaussian l in {0.5, 1, 2, 4},
  mu=1e-2, k estimated (Alg. 4) and capped at 4000, w=64, 1 or 32 RHS.
* ``clusters_3d``      n=200000, d=3: 80% from 3 isotropic normal clusters
  (centres U[0,1]^3, sigma 0.1, equal weights), 20% U[0,1]^3, shuffled;
  Matern-3/2 l=0.05, mu=1e-3, k=2000, w=50, 64 RHS.
* ``batched_512``      512 systems, n = floor(exp U[ln 256, ln 8192]),
  d uniform in {2..16}, N(0, I), Gaussian, l = median pairwise distance x
  exp U[ln 0.1, ln 10], mu = exp U[ln 1e-4, ln 1e-1], k = min(n//4, 1000),
  w = 32, 8 RHS each.
* ``serving_stream``   Poisson arrivals, n = floor(exp U[ln 1e3, ln 1e5]),
  d in {3, 8, 16}, kernel 50/50 Gaussian / Matern-3/2, l and mu as above,
  1..16 RHS.
* ``paper_cube_3d``    the setting of the paper's synthetic 3-D experiments
  (Sec. 5, Tables 1-2): n = 160,000 points U[0, n^(1/3)]^3, mu = 1e-4, one
  U[-0.5, 0.5] right-hand side, tol 1e-4; Gaussian l^2 and Matern-3/2 1/l
  taken from the tables' columns, w = 100 (the tables' FSAI with 100
  neighbours).  Seed 1006.

The median pairwise distance is exact (all i<j pairs, lower median) for
n <= 2048 and estimated from 10^5 seeded random pairs above that.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

GAUSSIAN = 0
MATERN32 = 1


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def uniform_points(n, d, seed, lo=0.0, hi=1.0):
    return rng(seed).uniform(lo, hi, size=(n, d))


def normal_points(n, d, seed):
    return rng(seed).standard_normal((n, d))


def rhs(n, nrhs, seed):
    """n x nrhs N(0,1), returned column-major (Fortran order)."""
    return np.asfortranarray(rng(seed).standard_normal((nrhs, n)).T)


@dataclass
class System:
    name: str
    X: np.ndarray              # n x d, row-major, float64
    B: np.ndarray              # n x nrhs, column-major, float64
    kernel: int
    l: float
    mu: float
    k: int                     # fixed k, or the cap when rank_mode == "estimate"
    w: int
    rank_mode: str = "fixed"   # "fixed" or "estimate" (Alg. 4)
    landmarks: str = "fps"     # "fps", "uniform" or "auto"
    fps_start: int = 0
    seed: int = 0
    extra: dict = field(default_factory=dict)

    @property
    def n(self):
        return self.X.shape[0]

    @property
    def d(self):
        return self.X.shape[1]

    @property
    def nrhs(self):
        return self.B.shape[1]


def median_pairwise_distance(X, seed, exact_limit=2048, samples=100_000):
    n = X.shape[0]
    if n <= exact_limit:
        G = X @ X.T
        sq = np.diag(G)
        D2 = np.maximum(sq[:, None] + sq[None, :] - 2.0 * G, 0.0)
        iu = np.triu_indices(n, 1)
        v = np.sqrt(np.sort(D2[iu]))
    else:
        g = rng(seed)
        i = g.integers(0, n, samples)
        j = g.integers(0, n - 1, samples)
        j = np.where(j >= i, j + 1, j)
        v = np.sort(np.sqrt(((X[i] - X[j]) ** 2).sum(1)))
    return float(v[(len(v) - 1) // 2])


def uniform_cube_3d(n=2000, seed=1001):
    g = rng(seed)
    X = g.uniform(0.0, 1.0, size=(n, 3))
    B = np.asfortranarray(g.standard_normal((1, n)).T)
    return System("uniform_cube_3d", X, B, GAUSSIAN, 0.1, 1e-4, min(200, n), 32)


def normal_8d(l=1.0, nrhs=32, n=50_000, seed=1002, k_max=4000, w=64):
    g = rng(seed)
    X = g.standard_normal((n, 8))
    B = np.asfortranarray(g.standard_normal((32, n)).T[:, :nrhs])
    return System("normal_8d", X, B, GAUSSIAN, float(l), 1e-2, k_max, w, rank_mode="estimate",
                  seed=seed)


def clusters_3d(n=200_000, nrhs=64, seed=1003, k=2000, w=50):
    g = rng(seed)
    nc = int(round(0.8 * n))
    centres = g.uniform(0.0, 1.0, size=(3, 3))
    lab = g.integers(0, 3, nc)
    Xc = centres[lab] + 0.1 * g.standard_normal((nc, 3))
    Xu = g.uniform(0.0, 1.0, size=(n - nc, 3))
    X = np.concatenate([Xc, Xu])[g.permutation(n)]
    B = np.asfortranarray(g.standard_normal((nrhs, n)).T)
    return System("clusters_3d", X, B, MATERN32, 0.05, 1e-3, k, w)


# the length-scale columns of the paper's Table 1 (a: Gaussian l^2, b: Matern-3/2 1/l)
PAPER_GAUSSIAN_L2 = (1000.0, 65.0, 60.0, 55.0, 50.0, 45.0, 40.0, 35.0, 30.0, 25.0, 0.1)
PAPER_MATERN_INV_L = (1.0, 0.065, 0.060, 0.055, 0.050, 0.045, 0.040, 0.035, 0.030, 0.025, 0.001)


def paper_cube_3d(n=160_000, seed=1006):
    """Points U[0, n^(1/3)]^3 and one U[-0.5, 0.5] right-hand side (Sec. 5)."""
    g = rng(seed)
    X = g.uniform(0.0, n ** (1.0 / 3.0), size=(n, 3))
    B = np.asfortranarray(g.uniform(-0.5, 0.5, size=(1, n)).T)
    return System("paper_cube_3d", X, B, GAUSSIAN, 1.0, 1e-4, 20000, 100, rank_mode="estimate",
                  seed=seed)


def _random_system(g, idx, n, d, kernel, nrhs, seed_base, name, w=32):
    sseed = seed_base * 1_000_000 + idx
    sg = rng(sseed)
    X = sg.standard_normal((n, d))
    B = np.asfortranarray(sg.standard_normal((nrhs, n)).T)
    med = median_pairwise_distance(X, sseed + 7)
    l = med * math.exp(g.uniform(math.log(0.1), math.log(10.0)))
    mu = math.exp(g.uniform(math.log(1e-4), math.log(1e-1)))
    return System(name, X, B, kernel, float(l), float(mu), min(n // 4, 1000), w, landmarks="auto",
                  seed=sseed)


def batched_512(count=512, seed=1004, nrhs=8, n_lo=256, n_hi=8192):
    """The batched workload; each system's points/RHS come from its own seed."""
    g = rng(seed)
    out = []
    for s in range(count):
        n = int(math.floor(math.exp(g.uniform(math.log(n_lo), math.log(n_hi)))))
        d = int(g.integers(2, 17))
        out.append(_random_system(g, s, n, d, GAUSSIAN, nrhs, seed, "batched_512"))
    return out


def serving_stream(count=10_000, seed=1005, rate=1.0, n_lo=1000, n_hi=100_000, materialize=False):
    """Request descriptors of the serving workload: arrival time (Poisson at
    ``rate`` per second), n, d, kernel, nrhs and the system seed.  Points and
    RHS are drawn on demand with ``serving_system``."""
    g = rng(seed)
    t = 0.0
    reqs = []
    for r in range(count):
        t += g.exponential(1.0 / rate)
        n = int(math.floor(math.exp(g.uniform(math.log(n_lo), math.log(n_hi)))))
        d = int(g.choice([3, 8, 16]))
        kernel = int(g.integers(0, 2))
        nrhs = int(g.integers(1, 17))
        lf = float(math.exp(g.uniform(math.log(0.1), math.log(10.0))))
        mu = float(math.exp(g.uniform(math.log(1e-4), math.log(1e-1))))
        reqs.append(dict(id=r, t=t, n=n, d=d, kernel=kernel, nrhs=nrhs, lfac=lf, mu=mu,
                         seed=seed * 1_000_000 + r))
    return reqs


def serving_system(req):
    sg = rng(req["seed"])
    X = sg.standard_normal((req["n"], req["d"]))
    B = np.asfortranarray(sg.standard_normal((req["nrhs"], req["n"])).T)
    med = median_pairwise_distance(X, req["seed"] + 7)
    return System("serving_stream", X, B, req["kernel"], med * req["lfac"], req["mu"],
                  min(req["n"] // 4, 1000), 32, landmarks="auto", seed=req["seed"])
