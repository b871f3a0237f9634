"""Host check of the three-term BF16 split of the apply's vector blocks.

The BF16 tensor-core W products of the mixed apply multiply a BF16 image of W
by the FP32 vector block written as three BF16 terms, x = b0 + b1 + b2, each
term rounded to nearest even from what the previous ones left.  BF16 keeps 8
significant bits and FP32's exponent range, so each remainder is exact in
FP32 and three terms carry all 24 bits of x for 2^-109 <= |x| < 3.39e38
(below, the last term is subnormal and less than 2^-125 is lost; above, the
first term rounds to infinity; neither is near any vector the apply sees):
the split loses nothing, and the
products of BF16 values (16 significant bits) are exact in the FP32
accumulator.  The only rounding of the vector side is therefore the FP32
accumulation itself.
"""
import numpy as np

from paper_2304_05460_gb300 import inputs

f32 = np.float32


def bf16_rn(x):
    """FP32 -> BF16 (as FP32 values), round to nearest even."""
    b = x.astype(f32).view(np.uint32)
    lsb = (b >> np.uint32(16)) & np.uint32(1)
    r = (b + np.uint32(0x7FFF) + lsb) & np.uint32(0xFFFF0000)
    return r.view(f32)


def split3(x):
    x = x.astype(f32)
    out = []
    for _ in range(3):
        b = bf16_rn(x)
        out.append(b)
        x = (x - b).astype(f32)
    return out, x


def test_three_bf16_terms_carry_fp32_exactly():
    g = inputs.rng(91)
    x = np.concatenate([
        g.standard_normal(200000),
        g.standard_normal(20000) * 1e30,
        g.standard_normal(20000) * 1e-30,
        np.ldexp(g.uniform(1, 2, 20000), g.integers(-120, 120, 20000)),
        [0.0, -0.0, 1.0, -1.0, 3.3e38, -3.3e38, 1.2e-38, 65504.0, 1.0 + 2.0 ** -23],
    ]).astype(f32)
    terms, rest = split3(x)
    for b in terms:
        assert np.all(b.view(np.uint32) & np.uint32(0xFFFF) == 0)     # BF16 values
    # exact while the last term stays a normal number (|x| >= 2^-109); below, the
    # subnormal last term drops less than 2^-125
    normal = (np.abs(x) >= 2.0 ** -109) | (x == 0)
    assert np.all(rest[normal] == 0)
    assert np.all(np.abs(rest[~normal]) < 2.0 ** -125)
    recon = (terms[0].astype(np.float64) + terms[1].astype(np.float64)
             + terms[2].astype(np.float64))
    assert np.array_equal(recon[normal], x[normal].astype(np.float64))


def test_two_terms_would_not_be_enough():
    x = inputs.rng(92).standard_normal(10000).astype(f32)
    b0 = bf16_rn(x)
    b1 = bf16_rn((x - b0).astype(f32))
    assert np.any((x - b0 - b1).astype(f32) != 0)


def test_bf16_products_exact_in_fp32():
    g = inputs.rng(93)
    a = bf16_rn(g.standard_normal(100000).astype(f32))
    b = bf16_rn(g.standard_normal(100000).astype(f32))
    assert np.array_equal((a * b).astype(np.float64), a.astype(np.float64) * b.astype(np.float64))
