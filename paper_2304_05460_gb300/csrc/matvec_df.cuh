// matvec_df.cuh -- FP64-accurate kernel matvec on the FP32 pipes.
//
// The FP64 residual b - (K + mu I) x of the mixed-precision solve needs
// about 1e-10 relative accuracy per product term; GB300's FP64 rate is 1/64
// of its FP32 rate.  Here every quantity is an unevaluated sum of two floats
// ("double-float", 48-bit significand) and every step is an error-free
// transformation: TwoSum (Knuth, TAOCP vol. 2, 4.2.2), Fast2Sum and the
// FMA-based TwoProduct (Dekker 1971).  The kernel value 2^-z is computed
// with a table-driven reduction (Tang 1989, ACM TOMS 15(2)):
// -z = m + j/64 + g with |g| <= 1/128, 2^-z = 2^m 2^(j/64) e^(g ln 2), the
// 64 table values 2^(j/64) and ln 2 carried as double-floats rounded from
// the host's FP64 values, and e^y = 1 + y + y^2/2 + y^3 P(y) from its Taylor
// series (|y| < 0.0055, so the cubic tail needs single precision only).
// Relative error of a kernel value is about 1e-14; sums are double-float.
#pragma once

#include <stdint.h>

namespace afn {

struct dfl {
    float h, l;
};

// Knuth's TwoSum: s + e == a + b exactly
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// Fast2Sum (|a| >= |b|)
__device__ __forceinline__ dfl fast_two_sum(float a, float b)
{
    dfl r;
    r.h = __fadd_rn(a, b);
    r.l = __fsub_rn(b, __fsub_rn(r.h, a));
    return r;
}

__device__ __forceinline__ dfl df_mul(dfl a, dfl b)
{
    const float p = __fmul_rn(a.h, b.h);
    float e = __fmaf_rn(a.h, b.h, -p);
    e = __fmaf_rn(a.h, b.l, e);
    e = __fmaf_rn(a.l, b.h, e);
    return fast_two_sum(p, e);
}

__device__ __forceinline__ dfl df_add(dfl a, dfl b)
{
    float s, e;
    two_sum(a.h, b.h, s, e);
    e = __fadd_rn(e, __fadd_rn(a.l, b.l));
    return fast_two_sum(s, e);
}

// constants of the exponential, set once per kernel launch from the host
struct DfExpTable {
    float t_h[64], t_l[64];     // 2^(j/64)
    float ln2_h, ln2_l;          // ln 2
    float log2e_h, log2e_l;      // log2 e
};

// 2^u for a double-float u <= 0 (0 below 2^-125, where the kernel value is
// negligible next to the unit diagonal)
__device__ __forceinline__ dfl df_exp2_neg(dfl u, const DfExpTable &T)
{
    dfl r{0.f, 0.f};
    if (!(u.h > -125.f)) return r;
    const float N = rintf(__fmul_rn(u.h, 64.f));
    const int ni = (int)N;
    const float gh = __fsub_rn(u.h, __fmul_rn(N, 0.015625f));   // exact (Sterbenz)
    float s, e;
    two_sum(gh, u.l, s, e);
    const dfl g = fast_two_sum(s, e);
    const int j = ni & 63;
    const int m = (ni - j) >> 6;
    const dfl y = df_mul(g, dfl{T.ln2_h, T.ln2_l});
    // e^y - 1 = y + y^2/2 + y^3 (1/6 + y/24 + y^2/120 + y^3/720)
    float q = __fmaf_rn(y.h, 1.f / 720.f, 1.f / 120.f);
    q = __fmaf_rn(q, y.h, 1.f / 24.f);
    q = __fmaf_rn(q, y.h, 1.f / 6.f);
    const float y3 = __fmul_rn(__fmul_rn(y.h, y.h), y.h);
    const float tail = __fmul_rn(q, y3);
    const float p2 = __fmul_rn(y.h, y.h);
    float p2e = __fmaf_rn(y.h, y.h, -p2);
    p2e = __fmaf_rn(__fmul_rn(2.f, y.h), y.l, p2e);
    dfl half_y2 = fast_two_sum(__fmul_rn(0.5f, p2), __fmul_rn(0.5f, p2e));
    dfl em1 = df_add(half_y2, dfl{tail, 0.f});
    em1 = df_add(y, em1);
    const dfl ey = df_add(dfl{1.f, 0.f}, em1);
    r = df_mul(dfl{T.t_h[j], T.t_l[j]}, ey);
    const float sc = __int_as_float((m + 127) << 23);   // 2^m, m >= -126
    r.h = __fmul_rn(r.h, sc);
    r.l = __fmul_rn(r.l, sc);
    return r;
}

// squared distance of prescaled double-float coordinates (row i in xi,
// point j at xj), summed over the DS dimensions in order
template <int DS>
__device__ __forceinline__ dfl df_dist2(const dfl (&xi)[DS], const float2 *xj)
{
    float zh = 0.f, zc = 0.f;
#pragma unroll
    for (int q = 0; q < DS; ++q) {
        const float2 b = xj[q];
        float s, e;
        two_sum(xi[q].h, -b.x, s, e);
        e = __fadd_rn(e, __fsub_rn(xi[q].l, b.y));
        const dfl dd = fast_two_sum(s, e);
        const float p = __fmul_rn(dd.h, dd.h);
        float pe = __fmaf_rn(dd.h, dd.h, -p);
        pe = __fmaf_rn(__fmul_rn(2.f, dd.h), dd.l, pe);
        float t;
        two_sum(zh, p, zh, t);
        zc = __fadd_rn(zc, __fadd_rn(t, pe));
    }
    return fast_two_sum(zh, zc);
}

// kernel value from the prescaled squared distance z:
//   Gaussian (coordinates x sqrt(log2 e)/l):  2^-z
//   Matern-3/2 (coordinates x sqrt(3)/l):     (1 + t) e^-t, t = sqrt(z)
template <int KER>
__device__ __forceinline__ dfl df_kernel(dfl z, const DfExpTable &T)
{
    if (KER == 0) return df_exp2_neg(dfl{-z.h, -z.l}, T);
    dfl t{0.f, 0.f};
    if (z.h > 0.f) {
        // t = sqrt(z): one Newton step on the single-precision root in
        // double-float (Karp and Markstein 1997)
        const float t0 = __fsqrt_rn(z.h);
        const float p = __fmul_rn(t0, t0);
        const float pe = __fmaf_rn(t0, t0, -p);
        const float rr = __fadd_rn(__fsub_rn(__fsub_rn(z.h, p), pe), z.l);
        t = fast_two_sum(t0, __fdiv_rn(rr, __fmul_rn(2.f, t0)));
    }
    const dfl u = df_mul(t, dfl{T.log2e_h, T.log2e_l});
    const dfl ex = df_exp2_neg(dfl{-u.h, -u.l}, T);
    return df_mul(df_add(dfl{1.f, 0.f}, t), ex);
}

}  // namespace afn
