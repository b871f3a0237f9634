"""Where the FP32 matvec's parity bar comes from: a host model of its arithmetic.

The mixed-precision matvec q = (K + mu I) p is checked on the GPU against the
FP64 oracle to 2e-5 of sum_j |K_ij p_j| + mu |p_i| per entry.  This file
replays the steps of that computation in IEEE FP32 with numpy and measures
the error they make by themselves, so that the bar can be read against it:

* points prescaled once, x~ = fl32(x s) (s = sqrt(log2 e) / l for the
  Gaussian, sqrt(3) / l for Matern-3/2), p rounded to FP32;
* r~^2 summed over the coordinates in FP32 (here with a separate multiply and
  add, one rounding more than the device's FMA);
* the kernel value from FP32 approximations of 2^x (and the square root for
  Matern), each given a random relative error of up to 2^-21 (2^-22 for the
  root) on top of correct rounding;
* K and p split into tf32 hi / lo words (round to nearest, ties away), the
  product formed as K_lo p_hi + K_hi p_lo + K_hi p_hi, eight points per
  accumulation step; the accumulator either rounds to nearest or truncates
  toward zero at every step (the tensor cores' accumulation is not specified
  beyond FP32, truncation is the worse case);
* blocks of 32 points folded into Kahan sums, split-K chunks of the point
  range summed in order, then mu p added.

With the modelled arithmetic the error stays below 1e-6 of the scale whether
the accumulator rounds or truncates (3e-7 at most on the configurations
below), so the bar leaves a margin of 20x over the modelled arithmetic for
what the model cannot reproduce bit for bit (the hardware's approximations
and its accumulation order inside one step).
"""
import math

import numpy as np
import pytest

import oracle
from paper_2304_05460_gb300 import inputs

f32 = np.float32
BAR = 2e-5           # the GPU parity bar of the FP32 matvec (tests/test_gpu_parity.py)


def _tf32_split(x):
    b = x.astype(f32).view(np.uint32)
    hi = ((b + np.uint32(0x1000)) & np.uint32(0xffffe000)).view(f32)
    r = (x - hi).astype(f32)                       # exact: hi is x rounded to 11 bits
    lo = ((r.view(np.uint32) + np.uint32(0x1000)) & np.uint32(0xffffe000)).view(f32)
    return hi, lo


def _round(x64, truncate):
    y = x64.astype(f32)
    if truncate:
        over = np.abs(y.astype(np.float64)) > np.abs(x64)
        y[over] = np.nextafter(y[over], f32(0))
    return y


def _approx(v64, rel, g):
    return (v64 * (1.0 + rel * g.uniform(-1.0, 1.0, v64.shape))).astype(f32)


def model_rows(X, ker, l, mu, P, rows, truncate=False, js=4, seed=0):
    """The modelled FP32 matvec on the given rows (float64 array rows x nrhs)."""
    g = np.random.default_rng(seed)
    n, d = X.shape
    s = 1.2011224087864498 / l if ker == oracle.GAUSSIAN else math.sqrt(3.0) / l
    Xs = (X * s).astype(f32)
    P32 = P.astype(f32)
    phi, plo = _tf32_split(P32)
    chunk = -(-n // js)
    out = np.zeros((len(rows), P.shape[1]))
    for a, i in enumerate(rows):
        u = (Xs[i][None, :] - Xs).astype(f32)
        r2 = np.zeros(n, f32)
        for t in range(d):
            r2 = (r2 + (u[:, t] * u[:, t]).astype(f32)).astype(f32)
        if ker == oracle.GAUSSIAN:
            K = _approx(np.exp2(-r2.astype(np.float64)), 2.0 ** -21, g)
        else:
            t_ = _approx(np.sqrt(r2.astype(np.float64)), 2.0 ** -22, g)
            arg = (t_ * f32(-1.4426950408889634)).astype(f32)
            e = _approx(np.exp2(arg.astype(np.float64)), 2.0 ** -21, g)
            K = ((f32(1) + t_).astype(f32) * e).astype(f32)
        Kh, Kl = _tf32_split(K)
        q = np.zeros(P.shape[1], f32)
        for c0 in range(0, n, chunk):
            c1 = min(n, c0 + chunk)
            acc = np.zeros(P.shape[1], f32)
            cmp = np.zeros(P.shape[1], f32)
            for b0 in range(c0, c1, 32):
                D = np.zeros(P.shape[1], f32)
                for k0 in range(b0, min(c1, b0 + 32), 8):
                    k1 = min(c1, k0 + 8)
                    for A, B in ((Kl, phi), (Kh, plo), (Kh, phi)):
                        # products of tf32 words are exact in FP64; one rounding per step
                        step = (A[k0:k1, None].astype(np.float64) * B[k0:k1]).sum(0)
                        D = _round(D.astype(np.float64) + step, truncate)
                y = (D - cmp).astype(f32)
                tot = (acc + y).astype(f32)
                cmp = ((tot - acc).astype(f32) - y).astype(f32)
                acc = tot
            q = (q + acc).astype(f32)
        out[a] = (q + (f32(mu) * P32[i]).astype(f32)).astype(f32)
    return out


def _rel_err(X, ker, l, mu, P, rows, truncate):
    q = model_rows(X, ker, l, mu, P, rows, truncate)
    ref = oracle.matvec_rows(X, ker, l, mu, P, rows).reshape(q.shape)
    scale = oracle.matvec_rows(X, ker, l, mu, np.abs(P), rows).reshape(q.shape)
    return float((np.abs(q - ref) / scale).max())


def test_tf32_split_reconstructs_to_2_pow_minus_22():
    x = np.concatenate([inputs.rng(1).standard_normal(4000), [0.0, 1.0, -1.0, 3.0e-30, 6.5e4]])
    x = x.astype(f32)
    hi, lo = _tf32_split(x)
    for w in (hi, lo):
        assert np.all(w.view(np.uint32) & np.uint32(0x1fff) == 0)     # 10 explicit mantissa bits
    err = np.abs(x.astype(np.float64) - hi.astype(np.float64) - lo.astype(np.float64))
    assert np.all(err <= 2.0 ** -22 * np.abs(x.astype(np.float64)))


@pytest.mark.parametrize("n,d,ker,nrhs", [(257, 3, oracle.GAUSSIAN, 1), (1000, 8, oracle.MATERN32, 3),
                                          (2049, 16, oracle.GAUSSIAN, 32), (1500, 2, oracle.MATERN32, 7),
                                          (777, 16, oracle.GAUSSIAN, 64)])
def test_modelled_error_far_below_the_bar(n, d, ker, nrhs):
    # the configurations of the GPU parity test of the FP32 matvec
    X = inputs.normal_points(n, d, 400 + n)
    P = inputs.rhs(n, nrhs, 401 + n)
    rows = np.arange(0, n, max(1, n // 24))
    l = 0.7 * math.sqrt(d)
    for truncate in (False, True):
        assert _rel_err(X, ker, l, 1e-2, P, rows, truncate) <= BAR / 20


@pytest.mark.parametrize("which", ["normal_8d", "clusters_3d"])
def test_modelled_error_at_full_size(which):
    # sampled rows of the full-size workloads the benchmark times (16 columns)
    if which == "normal_8d":
        s = inputs.normal_8d(l=2.0, nrhs=16)
        rows = np.arange(0, s.n, s.n // 4)
    else:
        s = inputs.clusters_3d(nrhs=16)
        rows = np.arange(0, s.n, s.n // 3)
    for truncate in (False, True):
        assert _rel_err(s.X, s.kernel, s.l, s.mu, s.B, rows, truncate) <= BAR / 20
