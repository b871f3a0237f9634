"""Host replay of the double-float kernel values of the FP64-accurate matvec.

The DF matvec forms each kernel value on the FP32 pipes as a double-float
(an unevaluated sum h + l of two floats): the squared distance of prescaled
double-float coordinates by TwoSum / TwoProduct steps, then 2^-z by a
table-driven reduction (-z = m + j/64 + g, 2^(j/64) from a 64-entry table,
e^(g ln 2) from its Taylor series) for the Gaussian, and t = sqrt(z) by one
Newton step followed by (1 + t) 2^(-t log2 e) for Matern-3/2.  This file
replays those steps in IEEE FP32 with numpy (an FMA emulated as one FP64
operation rounded to FP32) and measures them against 40-digit arithmetic
(mpmath), which fixes what the DF matvec's 1e-12 parity bar rests on:

* 2^-z: relative error below 2e-14 while 2^-z >= 2^-100; below that the low
  word enters FP32's subnormal range and only the absolute error stays tiny
  (below 1e-44); 0 from z = 125 on;
* Matern-3/2: absolute error below 2e-14 (the values lie in [0, 1]);
* the squared distance: relative error below 5e-14 of the exact distance of
  the double-float coordinates;
* a whole row of kernel values from FP64 points: sum_j |K~_ij - K_ij| |p_j|
  below 5e-14 of sum_j K_ij |p_j| + mu |p_i|, 20x inside the 1e-12 bar.
"""
import math

import numpy as np
import pytest

from paper_2304_05460_gb300 import inputs

mpmath = pytest.importorskip("mpmath")
mpmath.mp.dps = 40

f32, f64 = np.float32, np.float64
LN2 = 0.6931471805599453094
LOG2E = 1.4426950408889634074


def _fma(a, b, c):
    return (a.astype(f64) * b.astype(f64) + c.astype(f64)).astype(f32)


def _two_sum(a, b):
    s = (a + b).astype(f32)
    bb = (s - a).astype(f32)
    return s, ((a - (s - bb)).astype(f32) + (b - bb).astype(f32)).astype(f32)


def _fast_two_sum(a, b):
    h = (a + b).astype(f32)
    return h, (b - (h - a)).astype(f32)


def _df_mul(ah, al, bh, bl):
    p = (ah * bh).astype(f32)
    e = _fma(ah, bh, -p)
    e = _fma(ah, bl, e)
    e = _fma(al, bh, e)
    return _fast_two_sum(p, e)


def _df_add(ah, al, bh, bl):
    s, e = _two_sum(ah, bh)
    return _fast_two_sum(s, (e + (al + bl).astype(f32)).astype(f32))


def _split(v):
    h = np.asarray(v, dtype=f64).astype(f32)
    return h, (np.asarray(v, dtype=f64) - h).astype(f32)


_TH, _TL = _split(np.exp2(np.arange(64) / 64.0))
_LN2H, _LN2L = _split(LN2)
_L2EH, _L2EL = _split(LOG2E)


def df_exp2_neg(uh, ul):
    """2^u for a double-float u <= 0 (0 below -125)."""
    N = np.rint((uh * f32(64)).astype(f32))
    ni = N.astype(np.int64)
    gh = (uh - (N * f32(0.015625)).astype(f32)).astype(f32)
    gh, gl = _fast_two_sum(*_two_sum(gh, ul))
    j = ni & 63
    m = (ni - j) >> 6
    one = np.ones_like(gh)
    yh, yl = _df_mul(gh, gl, one * _LN2H, one * _LN2L)
    q = _fma(yh, one * f32(1 / 720), one * f32(1 / 120))
    q = _fma(q, yh, one * f32(1 / 24))
    q = _fma(q, yh, one * f32(1 / 6))
    tail = (q * ((yh * yh).astype(f32) * yh).astype(f32)).astype(f32)
    p2 = (yh * yh).astype(f32)
    p2e = _fma((f32(2) * yh).astype(f32), yl, _fma(yh, yh, -p2))
    hh, hl = _fast_two_sum((f32(0.5) * p2).astype(f32), (f32(0.5) * p2e).astype(f32))
    eh, el = _df_add(hh, hl, tail, np.zeros_like(tail))
    eh, el = _df_add(yh, yl, eh, el)
    eh, el = _df_add(one, np.zeros_like(one), eh, el)
    rh, rl = _df_mul(_TH[j], _TL[j], eh, el)
    sc = np.ldexp(np.ones(rh.shape), m).astype(f32)
    rh, rl = (rh * sc).astype(f32), (rl * sc).astype(f32)
    dead = ~(uh > f32(-125))
    rh[dead] = 0
    rl[dead] = 0
    return rh, rl


def df_matern(zh, zl):
    """(1 + t) 2^(-t log2 e), t = sqrt(z) by one Newton step in double-float."""
    th = np.zeros_like(zh)
    tl = np.zeros_like(zh)
    pos = zh > 0
    t0 = np.sqrt(zh[pos]).astype(f32)
    p = (t0 * t0).astype(f32)
    rr = (((zh[pos] - p).astype(f32) - _fma(t0, t0, -p)).astype(f32) + zl[pos]).astype(f32)
    th[pos], tl[pos] = _fast_two_sum(t0, (rr / (f32(2) * t0).astype(f32)).astype(f32))
    one = np.ones_like(th)
    uh, ul = _df_mul(th, tl, one * _L2EH, one * _L2EL)
    eh, el = df_exp2_neg(-uh, -ul)
    ah, al = _df_add(one, np.zeros_like(one), th, tl)
    return _df_mul(ah, al, eh, el)


def df_dist2(xih, xil, Xjh, Xjl):
    """Squared distance of double-float coordinates, dimensions in order."""
    zh = np.zeros(Xjh.shape[0], f32)
    zc = np.zeros_like(zh)
    for q in range(Xjh.shape[1]):
        s, e = _two_sum(np.full_like(zh, xih[q]), -Xjh[:, q])
        dh, dl = _fast_two_sum(s, (e + (xil[q] - Xjl[:, q]).astype(f32)).astype(f32))
        p = (dh * dh).astype(f32)
        pe = _fma((f32(2) * dh).astype(f32), dl, _fma(dh, dh, -p))
        zh, t = _two_sum(zh, p)
        zc = (zc + (t + pe).astype(f32)).astype(f32)
    return _fast_two_sum(zh, zc)


def _val(h, l):
    return h.astype(f64) + l.astype(f64)


def _mp(h, l):
    return mpmath.mpf(float(h)) + mpmath.mpf(float(l))


def test_exp2_of_double_float_arguments():
    g = inputs.rng(71)
    z = np.concatenate([g.uniform(0, 1, 1500), g.uniform(1, 100, 1500), g.uniform(100, 125, 400),
                        [0.0, 1e-30, 0.5, 1.0, 64.0, 99.99]])
    zh, zl = _split(z)
    rh, rl = df_exp2_neg(-zh, -zl)
    got = _val(rh, rl)
    exact = np.array([float(mpmath.power(2, -_mp(a, b))) for a, b in zip(zh, zl)])
    small = z <= 100
    assert np.all(np.abs(got - exact)[small] <= 2e-14 * exact[small])
    assert np.all(np.abs(got - exact)[~small] <= 1e-44)
    dead = df_exp2_neg(np.array([-125.0, -300.0], f32), np.zeros(2, f32))
    assert np.all(dead[0] == 0) and np.all(dead[1] == 0)


def test_matern_value_absolute_error():
    g = inputs.rng(72)
    z = np.concatenate([g.uniform(0, 1, 1500), g.uniform(1, 100, 1500), g.uniform(100, 4000, 800),
                        [0.0, 1e-20, 1.0, 3.0]])
    zh, zl = _split(z)
    got = _val(*df_matern(zh, zl))

    def exact(a, b):
        t = mpmath.sqrt(_mp(a, b))
        return float((1 + t) * mpmath.exp(-t))
    ref = np.array([exact(a, b) for a, b in zip(zh, zl)])
    assert np.all(np.abs(got - ref) <= 2e-14)
    assert got[-4] == 1.0


@pytest.mark.parametrize("d,scale", [(3, 1.0), (8, 1.0), (16, 1.0), (3, 30.0)])
def test_squared_distance(d, scale):
    X = inputs.normal_points(200, d, 73 + d) * scale
    Xh, Xl = _split(X)
    for i in range(0, 200, 25):
        got = _val(*df_dist2(Xh[i], Xl[i], Xh, Xl))
        for j in range(200):
            ex = mpmath.fsum((_mp(Xh[i, q], Xl[i, q]) - _mp(Xh[j, q], Xl[j, q])) ** 2
                             for q in range(d))
            assert abs(mpmath.mpf(float(got[j])) - ex) <= 5e-14 * ex


@pytest.mark.parametrize("kernel", [0, 1])
def test_row_of_kernel_values_from_fp64_points(kernel):
    # prescaled as the device does: x * sqrt(log2 e) / l (Gaussian) or x * sqrt(3) / l
    # (Matern) in FP64, split into double-floats; exact values from the FP64 points
    n, d, l, mu = 160, 8, 2.0, 1e-2
    X = inputs.normal_points(n, d, 74)
    P = np.abs(inputs.rhs(n, 1, 75)[:, 0])
    s = (1.2011224087864498 if kernel == 0 else 1.7320508075688772) / l
    Xh, Xl = _split(X * s)
    for i in range(0, n, 16):
        zh, zl = df_dist2(Xh[i], Xl[i], Xh, Xl)
        K = _val(*(df_exp2_neg(-zh, -zl) if kernel == 0 else df_matern(zh, zl)))
        ref = np.empty(n)
        for j in range(n):
            r2 = mpmath.fsum((mpmath.mpf(float(X[i, q])) - mpmath.mpf(float(X[j, q]))) ** 2
                             for q in range(d))
            if kernel == 0:
                ref[j] = float(mpmath.exp(-r2 / l ** 2))
            else:
                t = mpmath.sqrt(3 * r2) / l
                ref[j] = float((1 + t) * mpmath.exp(-t))
        err = float(np.sum(np.abs(K - ref) * P))
        scale = float(np.sum(ref * P) + mu * P[i])
        assert err <= 5e-14 * scale
