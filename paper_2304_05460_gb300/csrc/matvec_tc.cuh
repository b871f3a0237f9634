// matvec_tc.cuh -- the tensor-core tile of the FP32 kernel matvec, shared by
// the single-system kernel (matvec.cu) and the grouped multi-system kernel
// (batch.cu).
#pragma once

#include "afn_device.cuh"

namespace afn {

// --------------------------------------------------------------------------
// Tensor-core variant for 8, 16 or 32 right-hand sides.  The kernel-matrix
// block K[i, j] (16 rows x 8 points) is evaluated on the FP32 pipes directly
// into the A-fragment registers of mma.m16n8k8 (tf32), and the contraction
// with the p tile runs on the tensor cores in three tf32 passes
// (K_hi p_hi + K_hi p_lo + K_lo p_hi, each operand split as x = hi + lo with
// hi = tf32(x), lo = tf32(x - hi)), which keeps single-precision accuracy.
// A warp owns 16 rows; a CTA owns 128 rows and one j-chunk; point and p
// tiles (64 points) are staged in shared memory with bank-conflict-free
// strides.  Fragment layouts (PTX ISA, mma.m16n8k8 .tf32): with g = lane/4,
// t = lane%4, A holds (g,t) (g+8,t) (g,t+4) (g+8,t+4); B holds (t,g) (t+4,g);
// C holds (g,2t) (g,2t+1) (g+8,2t) (g+8,2t+1).
// --------------------------------------------------------------------------
__device__ __forceinline__ uint32_t tf32_bits(float x)
{
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

#ifndef AFN_TC_MINB
#define AFN_TC_MINB 3
#endif
#ifndef AFN_TC_FOLD
#define AFN_TC_FOLD 2
#endif
#ifndef AFN_TC_KAHAN
#define AFN_TC_KAHAN 1
#endif
static constexpr int TC_FOLD = AFN_TC_FOLD;        // blocks of 8 points per accumulator fold
static constexpr bool TC_KAHAN = AFN_TC_KAHAN != 0;

// x = hi + lo with hi, lo tf32 (10-bit mantissa) values, each rounded to
// nearest (ties away from zero): adding half a unit of the 13 dropped bits
// and masking them is that rounding for finite inputs.
__device__ __forceinline__ void tf32_split(float x, uint32_t &hi, uint32_t &lo)
{
#ifdef AFN_TC_CVT_SPLIT
    hi = tf32_bits(x);
    lo = tf32_bits(x - __uint_as_float(hi));
#else
    hi = (__float_as_uint(x) + 0x1000u) & 0xffffe000u;
    lo = (__float_as_uint(x - __uint_as_float(hi)) + 0x1000u) & 0xffffe000u;
#endif
}

__device__ __forceinline__ void mma_tf32(float (&c)[4], uint32_t a0, uint32_t a1, uint32_t a2,
                                         uint32_t a3, uint32_t b0, uint32_t b1)
{
    asm volatile("mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, "
                 "{%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
                 : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
                 : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

static constexpr int TCR = 128;   // rows per CTA (8 warps x 16)
static constexpr int TCJ = 64;    // points per staged tile

// PS: shared-memory stride of a staged p row, t*PS distinct mod 32 by 8s
template <int NB> struct TcPS { static constexpr int v = (NB == 1) ? 8 : (NB == 2 ? 24 : 40); };

// Sums sum_{j in [j0, j1)} K(x_i, x_j) p_j for the 16 rows of each warp of a
// 256-thread CTA (rows row0 + warp*16 + {g, g+8}), NB groups of 8 columns of
// p (column-major, leading dimension ldp).  xsd, phi, plo are the CTA's
// staging buffers: TCJ*(DS+2) f2_t and TCJ*TcPS<NB>::v words each.  All
// threads of the CTA must call it together.  On return acc[b][.] holds the
// C-fragment (g,2t) (g,2t+1) (g+8,2t) (g+8,2t+1) of column group b.
template <int DS, int NB, int KER>
__device__ __forceinline__ void mv32tc_rows(const float *__restrict__ Xs, int64_t n,
                                            const float *__restrict__ P, int64_t ldp,
                                            int64_t row0, int64_t j0, int64_t j1, f2_t *xsd,
                                            uint32_t *phi, uint32_t *plo, float (&acc)[NB][4])
{
    constexpr int NR = NB * 8;
    constexpr int PS = TcPS<NB>::v;
    constexpr int DSP = DS + 2;                                 // f2 stride of a point row
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = lane >> 2, t = lane & 3;
    const int64_t ia = row0 + warp * 16 + g;
    const int64_t ib = ia + 8;
    f2_t xi[DS];   // (x_ia[q], x_ib[q])
#pragma unroll
    for (int q = 0; q < DS; ++q)
        xi[q] = f2_pack(ia < n ? Xs[ia * DS + q] : 0.f, ib < n ? Xs[ib * DS + q] : 0.f);
    float cmp[TC_KAHAN ? NB : 1][4];
#pragma unroll
    for (int b = 0; b < NB; ++b)
#pragma unroll
        for (int r = 0; r < 4; ++r) acc[b][r] = 0.f;
#pragma unroll
    for (int b = 0; b < (TC_KAHAN ? NB : 1); ++b)
#pragma unroll
        for (int r = 0; r < 4; ++r) cmp[b][r] = 0.f;

    for (int64_t jt = j0; jt < j1; jt += TCJ) {
        __syncthreads();
        for (int e = threadIdx.x; e < TCJ * DS; e += 256) {
            int jj = e / DS, q = e % DS;
            int64_t j = jt + jj;
            float v = (j < j1) ? Xs[j * DS + q] : 0.f;
            xsd[jj * DSP + q] = f2_pack(v, v);
        }
        for (int e = threadIdx.x; e < TCJ * NR / 4; e += 256) {
            int jj = e % TCJ, c4 = e / TCJ;
            int64_t j = jt + jj;
            uint4 h4, l4;
            tf32_split(j < j1 ? P[(4 * c4 + 0) * ldp + j] : 0.f, h4.x, l4.x);
            tf32_split(j < j1 ? P[(4 * c4 + 1) * ldp + j] : 0.f, h4.y, l4.y);
            tf32_split(j < j1 ? P[(4 * c4 + 2) * ldp + j] : 0.f, h4.z, l4.z);
            tf32_split(j < j1 ? P[(4 * c4 + 3) * ldp + j] : 0.f, h4.w, l4.w);
            *reinterpret_cast<uint4 *>(phi + jj * PS + 4 * c4) = h4;
            *reinterpret_cast<uint4 *>(plo + jj * PS + 4 * c4) = l4;
        }
        __syncthreads();
        float tac[NB][4];
#pragma unroll
        for (int b = 0; b < NB; ++b)
#pragma unroll
            for (int r = 0; r < 4; ++r) tac[b][r] = 0.f;
#pragma unroll
        for (int kb = 0; kb < TCJ / 8; ++kb) {
            const f2_t *xa = xsd + (kb * 8 + t) * DSP;
            const f2_t *xb = xsd + (kb * 8 + t + 4) * DSP;
            f2_t ra = 0ull, rb = 0ull;
            // two coordinates per 16-byte shared-memory load (rows are
            // 16-byte aligned: DSP is even), half the wavefronts of 8-byte loads
#pragma unroll
            for (int q = 0; q < DS; q += 2) {
                const ulonglong2 va = *reinterpret_cast<const ulonglong2 *>(xa + q);
                const ulonglong2 vb = *reinterpret_cast<const ulonglong2 *>(xb + q);
                f2_t u = f2_sub(xi[q], va.x);
                ra = f2_fma(u, u, ra);
                u = f2_sub(xi[q], vb.x);
                rb = f2_fma(u, u, rb);
                u = f2_sub(xi[q + 1], va.y);
                ra = f2_fma(u, u, ra);
                u = f2_sub(xi[q + 1], vb.y);
                rb = f2_fma(u, u, rb);
            }
            float r_aa, r_ba, r_ab, r_bb;   // (row ia|ib, column t|t+4)
            f2_unpack(ra, r_aa, r_ba);
            f2_unpack(rb, r_ab, r_bb);
            uint32_t ah0, al0, ah1, al1, ah2, al2, ah3, al3;
            tf32_split(kernel32_scaled<KER>(r_aa), ah0, al0);   // (g,   t)
            tf32_split(kernel32_scaled<KER>(r_ba), ah1, al1);   // (g+8, t)
            tf32_split(kernel32_scaled<KER>(r_ab), ah2, al2);   // (g,   t+4)
            tf32_split(kernel32_scaled<KER>(r_bb), ah3, al3);   // (g+8, t+4)
            const uint32_t *ph0 = phi + (kb * 8 + t) * PS + g;
            const uint32_t *ph1 = phi + (kb * 8 + t + 4) * PS + g;
            const uint32_t *pl0 = plo + (kb * 8 + t) * PS + g;
            const uint32_t *pl1 = plo + (kb * 8 + t + 4) * PS + g;
#pragma unroll
            for (int b = 0; b < NB; ++b) {
                const uint32_t bh0 = ph0[b * 8], bh1 = ph1[b * 8];
                const uint32_t bl0 = pl0[b * 8], bl1 = pl1[b * 8];
                // small cross terms first, then the leading product
                mma_tf32(tac[b], al0, al1, al2, al3, bh0, bh1);
                mma_tf32(tac[b], ah0, ah1, ah2, ah3, bl0, bl1);
                mma_tf32(tac[b], ah0, ah1, ah2, ah3, bh0, bh1);
            }
            // The tensor-core accumulator is not rounded to nearest; folding
            // it into the FP32 running sum every TC_FOLD blocks of 8 points
            // keeps its error from growing over the whole j range.
            if ((kb + 1) % TC_FOLD == 0) {
#pragma unroll
                for (int b = 0; b < NB; ++b)
#pragma unroll
                    for (int r = 0; r < 4; ++r) {
                        if constexpr (TC_KAHAN) {
                            float y = tac[b][r] - cmp[b][r];
                            float s = acc[b][r] + y;
                            cmp[b][r] = (s - acc[b][r]) - y;
                            acc[b][r] = s;
                        } else {
                            acc[b][r] += tac[b][r];
                        }
                        tac[b][r] = 0.f;
                    }
            }
        }
    }
}

}  // namespace afn
