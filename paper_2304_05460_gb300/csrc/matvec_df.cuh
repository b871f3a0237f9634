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
// 2^-z is within 2e-14 relative while it is above 2^-100 (below that the low
// word is subnormal and only the absolute error stays below 1e-44), the
// Matern value within 2e-14 absolute, the squared distance within 5e-14
// relative; sums are double-float.
#pragma once

#include <stdint.h>

#include "afn_device.cuh"

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

// constants of the exponential, set once per kernel launch from the host
struct DfExpTable {
    float t_h[64], t_l[64];     // 2^(j/64)
    float ln2_h, ln2_l;          // ln 2
    float log2e_h, log2e_l;      // log2 e
};

// ---- two values per instruction --------------------------------------------
// Every operation below acts on two independent values at once with
// Blackwell's packed f32x2 add / sub / mul / fma (low half = first value);
// each half is rounded exactly as the scalar .rn operation would be, so the
// halves are the scalar results bit for bit.
struct dfl2 {
    f2_t h, l;
};

__device__ __forceinline__ f2_t f2_mul(f2_t a, f2_t b)
{
    f2_t d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

__device__ __forceinline__ f2_t f2_neg(f2_t a) { return a ^ 0x8000000080000000ull; }

__device__ __forceinline__ f2_t f2_splat(float v) { return f2_pack(v, v); }

__device__ __forceinline__ void two_sum2(f2_t a, f2_t b, f2_t &s, f2_t &e)
{
    s = f2_add(a, b);
    const f2_t bb = f2_sub(s, a);
    e = f2_add(f2_sub(a, f2_sub(s, bb)), f2_sub(b, bb));
}

__device__ __forceinline__ dfl2 fast_two_sum2(f2_t a, f2_t b)
{
    dfl2 r;
    r.h = f2_add(a, b);
    r.l = f2_sub(b, f2_sub(r.h, a));
    return r;
}

__device__ __forceinline__ dfl2 df_mul2(dfl2 a, dfl2 b)
{
    const f2_t p = f2_mul(a.h, b.h);
    f2_t e = f2_fma(a.h, b.h, f2_neg(p));
    e = f2_fma(a.h, b.l, e);
    e = f2_fma(a.l, b.h, e);
    return fast_two_sum2(p, e);
}

__device__ __forceinline__ dfl2 df_add2(dfl2 a, dfl2 b)
{
    f2_t s, e;
    two_sum2(a.h, b.h, s, e);
    e = f2_add(e, f2_add(a.l, b.l));
    return fast_two_sum2(s, e);
}

// 2^u for double-float u <= 0, two values (0 below 2^-125, where the kernel
// value is negligible next to the unit diagonal): -u = m + j/64 + g with
// |g| <= 1/128, 2^u = 2^m 2^(j/64) e^(g ln 2)
__device__ __forceinline__ dfl2 df_exp2_neg2(dfl2 u, const DfExpTable &T)
{
    float uh0, uh1;
    f2_unpack(u.h, uh0, uh1);
    const float N0 = rintf(__fmul_rn(uh0, 64.f)), N1 = rintf(__fmul_rn(uh1, 64.f));
    const int ni0 = (int)N0, ni1 = (int)N1;
    const f2_t gh = f2_sub(u.h, f2_mul(f2_pack(N0, N1), f2_splat(0.015625f)));   // exact (Sterbenz)
    f2_t s, e;
    two_sum2(gh, u.l, s, e);
    const dfl2 g = fast_two_sum2(s, e);
    const int j0 = ni0 & 63, j1 = ni1 & 63;
    const int m0 = (ni0 - j0) >> 6, m1 = (ni1 - j1) >> 6;
    const dfl2 y = df_mul2(g, dfl2{f2_splat(T.ln2_h), f2_splat(T.ln2_l)});
    // e^y - 1 = y + y^2/2 + y^3 (1/6 + y/24 + y^2/120 + y^3/720)
    f2_t q = f2_fma(y.h, f2_splat(1.f / 720.f), f2_splat(1.f / 120.f));
    q = f2_fma(q, y.h, f2_splat(1.f / 24.f));
    q = f2_fma(q, y.h, f2_splat(1.f / 6.f));
    const f2_t y3 = f2_mul(f2_mul(y.h, y.h), y.h);
    const f2_t tail = f2_mul(q, y3);
    const f2_t p2 = f2_mul(y.h, y.h);
    f2_t p2e = f2_fma(y.h, y.h, f2_neg(p2));
    p2e = f2_fma(f2_mul(f2_splat(2.f), y.h), y.l, p2e);
    const dfl2 half_y2 = fast_two_sum2(f2_mul(f2_splat(0.5f), p2), f2_mul(f2_splat(0.5f), p2e));
    dfl2 em1 = df_add2(half_y2, dfl2{tail, 0ull});
    em1 = df_add2(y, em1);
    const dfl2 ey = df_add2(dfl2{f2_splat(1.f), 0ull}, em1);
    dfl2 r = df_mul2(dfl2{f2_pack(T.t_h[j0], T.t_h[j1]), f2_pack(T.t_l[j0], T.t_l[j1])}, ey);
    const f2_t sc = f2_pack(__int_as_float((m0 + 127) << 23), __int_as_float((m1 + 127) << 23));
    r.h = f2_mul(r.h, sc);
    r.l = f2_mul(r.l, sc);
    // 0 below 2^-125 (the scalar form's early return)
    float rh0, rh1, rl0, rl1;
    f2_unpack(r.h, rh0, rh1);
    f2_unpack(r.l, rl0, rl1);
    if (!(uh0 > -125.f)) rh0 = rl0 = 0.f;
    if (!(uh1 > -125.f)) rh1 = rl1 = 0.f;
    return dfl2{f2_pack(rh0, rh1), f2_pack(rl0, rl1)};
}

// squared distance of prescaled double-float coordinates, summed over the DS
// dimensions in order, for the row point xi and two points j0, j1 whose
// coordinates come as packed pairs: xj[q] = {h(j0), h(j1), l(j0), l(j1)}
template <int DS>
__device__ __forceinline__ dfl2 df_dist2_2(const dfl (&xi)[DS], const float4 *xj)
{
    f2_t zh = 0ull, zc = 0ull;
#pragma unroll
    for (int q = 0; q < DS; ++q) {
        const float4 b = xj[q];
        f2_t s, e;
        two_sum2(f2_splat(xi[q].h), f2_neg(f2_pack(b.x, b.y)), s, e);
        e = f2_add(e, f2_sub(f2_splat(xi[q].l), f2_pack(b.z, b.w)));
        const dfl2 dd = fast_two_sum2(s, e);
        const f2_t p = f2_mul(dd.h, dd.h);
        f2_t pe = f2_fma(dd.h, dd.h, f2_neg(p));
        pe = f2_fma(f2_mul(f2_splat(2.f), dd.h), dd.l, pe);
        f2_t t;
        two_sum2(zh, p, zh, t);
        zc = f2_add(zc, f2_add(t, pe));
    }
    return fast_two_sum2(zh, zc);
}

// kernel value from the prescaled squared distance z, two values:
//   Gaussian (coordinates x sqrt(log2 e)/l):  2^-z
//   Matern-3/2 (coordinates x sqrt(3)/l):     (1 + t) e^-t, t = sqrt(z) by one
//   Newton step on the single-precision root in double-float (Karp and
//   Markstein 1997)
template <int KER>
__device__ __forceinline__ dfl2 df_kernel2(dfl2 z, const DfExpTable &T)
{
    if (KER == 0) return df_exp2_neg2(dfl2{f2_neg(z.h), f2_neg(z.l)}, T);
    float zh0, zh1, zl0, zl1;
    f2_unpack(z.h, zh0, zh1);
    f2_unpack(z.l, zl0, zl1);
    // t = sqrt(z): one Newton step on the single-precision root (per value)
    float th[2] = {0.f, 0.f}, tl[2] = {0.f, 0.f};
    const float zh_[2] = {zh0, zh1}, zl_[2] = {zl0, zl1};
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        if (zh_[h] > 0.f) {
            const float t0 = __fsqrt_rn(zh_[h]);
            const float p = __fmul_rn(t0, t0);
            const float pe = __fmaf_rn(t0, t0, -p);
            const float rr = __fadd_rn(__fsub_rn(__fsub_rn(zh_[h], p), pe), zl_[h]);
            const dfl t = fast_two_sum(t0, __fdiv_rn(rr, __fmul_rn(2.f, t0)));
            th[h] = t.h;
            tl[h] = t.l;
        }
    }
    const dfl2 t{f2_pack(th[0], th[1]), f2_pack(tl[0], tl[1])};
    const dfl2 u = df_mul2(t, dfl2{f2_splat(T.log2e_h), f2_splat(T.log2e_l)});
    const dfl2 ex = df_exp2_neg2(dfl2{f2_neg(u.h), f2_neg(u.l)}, T);
    return df_mul2(df_add2(dfl2{f2_splat(1.f), 0ull}, t), ex);
}

}  // namespace afn
