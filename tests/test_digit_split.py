"""Host check of the digit splitting that makes the double-float matvec's sum
exact on the BF16 tensor cores: the steps of the device code, replayed in
IEEE FP32 / FP64 with numpy, on random and edge-case values.

Kernel values v = h + l (a double-float in [0, 1]) are split into eight
digits a_s with v = sum_s a_s 2^(-7-8s) + remainder; p values into eight
digits b_t of p 2^(-E) (2^E > max |p|).  The exactness argument needs every
digit to be an integer of magnitude at most 256 (so exact in BF16; the bound
used for the accumulators is 192 for a and 128 for b) and the remainders to
be below 2^-64 (a) and 2^-56 (b)."""
from fractions import Fraction

import numpy as np

f32 = np.float32


def _round_to(r, c):
    # nearest multiple of g = c / (1.5 * 2^23): (r + c) - c in FP32
    return f32(f32(r + c) - c)


def _two_sum(a, b):
    s = f32(a + b)
    bb = f32(s - a)
    return s, f32(f32(a - f32(s - bb)) + f32(b - bb))


def k_digits(h, l):
    """The device's digit extraction of a double-float kernel value (FP32 steps)."""
    r, rl = f32(h), f32(l)
    d = []
    for s, (c, scale) in enumerate([(2.0 ** 16 * 1.5, 2.0 ** 7), (2.0 ** 8 * 1.5, 2.0 ** 15),
                                    (1.5, 2.0 ** 23), (2.0 ** -8 * 1.5, 2.0 ** 31),
                                    (2.0 ** -16 * 1.5, 2.0 ** 39), (2.0 ** -24 * 1.5, 2.0 ** 47),
                                    (2.0 ** -32 * 1.5, 2.0 ** 55), (2.0 ** -40 * 1.5, 2.0 ** 63)]):
        if s in (3, 6):
            r, rl = _two_sum(r, rl)
        src = f32(r + rl) if s == 7 else r
        a = _round_to(src, f32(c))
        if s < 7:
            r = f32(r - a)
        d.append(float(a) * scale)
    return d


def p_digits(p, E):
    """The device's digit extraction of an FP64 value p with 2^E > |p| (FP64 steps)."""
    w = np.ldexp(np.float64(p), 7 - E)
    d = []
    for _ in range(8):
        t = np.rint(w)
        w = (w - t) * 256.0
        d.append(float(t))
    return d


def _dfl(x):
    h = f32(x)
    return h, f32(np.float64(x) - np.float64(h))


def test_kernel_value_digits():
    g = np.random.default_rng(5)
    xs = list(g.random(4000)) + list(np.exp(-g.random(2000) * 80.0)) + [
        0.0, 1.0, 2.0 ** -125, 2.0 ** -64, 2.0 ** -40, 0.5, 1.0 - 2.0 ** -24, 1.0 - 2.0 ** -40,
        0.99999, 1.0 / 3.0]
    for x in xs:
        h, l = _dfl(x)
        d = k_digits(h, l)
        for s, a in enumerate(d):
            assert a == int(a), (x, s, a)
            assert abs(a) <= (192 if s in (3, 6) else 128), (x, s, a)
        v = Fraction(float(h)) + Fraction(float(l))
        rec = sum(Fraction(int(a)) * Fraction(1, 2 ** (7 + 8 * s)) for s, a in enumerate(d))
        assert abs(v - rec) <= Fraction(1, 2 ** 64), (x, float(v - rec))


def test_p_digits():
    g = np.random.default_rng(6)
    for scale in (1e-280, 1e-8, 1.0, 3.0, 1e6, 1e280):
        p = g.standard_normal(3000) * scale
        m = float(np.abs(p).max())
        E = int(np.frexp(m)[1])
        assert 2.0 ** E > m
        for x in list(p[:500]) + [p[np.argmax(np.abs(p))], 0.0]:
            d = p_digits(x, E)
            assert all(t == int(t) and abs(t) <= 128 for t in d), (x, d)
            rec = sum(Fraction(int(t)) * Fraction(1, 2 ** (7 + 8 * s)) for s, t in enumerate(d))
            err = Fraction(float(np.ldexp(np.float64(x), -E))) - rec
            assert abs(err) <= Fraction(1, 2 ** 56), (x, float(err))


def test_accumulator_bound():
    # per 32-point block, D_q sums at most 8 products of |a| <= 192 and |b| <= 128: an
    # integer below 2^23, so the FP32 accumulation of the BF16 products is exact
    assert 8 * 32 * 192 * 128 < 2 ** 23
