// matvec_tc.cuh -- the mma.sync tensor-core tile of the FP32 kernel matvec,
// used by the single-system kernel for 8-column pieces (16 and 32 columns
// run on the tcgen05 kernel of matvec_umma.cuh) and by the grouped
// multi-system kernel; also the tf32
// split and the staging helpers (mbarriers, bulk copies) both tiles share.
#pragma once

#include "afn_device.cuh"

namespace afn {

// --------------------------------------------------------------------------
// Tensor-core tile for 8, 16 or 32 right-hand sides.  The kernel-matrix
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
static constexpr int TC_MINB = 3;                  // resident CTAs per SM of the mma.sync tile
static constexpr int TC_FOLD = 2;                  // blocks of 8 points per accumulator fold
static_assert(TC_FOLD >= 1 && 8 % TC_FOLD == 0, "a fold chunk must not cross a staged tile");
static constexpr bool TC_KAHAN = true;             // accumulator folds are Kahan sums

// x = hi + lo with hi, lo tf32 (10-bit mantissa) values, each rounded to
// nearest (ties away from zero): adding half a unit of the 13 dropped bits
// and masking them is that rounding for finite inputs.
__device__ __forceinline__ void tf32_split(float x, uint32_t &hi, uint32_t &lo)
{
    hi = (__float_as_uint(x) + 0x1000u) & 0xffffe000u;
    lo = (__float_as_uint(x - __uint_as_float(hi)) + 0x1000u) & 0xffffe000u;
}

__device__ __forceinline__ void mma_tf32(float (&c)[4], uint32_t a0, uint32_t a1, uint32_t a2,
                                         uint32_t a3, uint32_t b0, uint32_t b1)
{
    asm volatile("mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, "
                 "{%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
                 : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
                 : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// c = A B (the accumulator input is zero: no registers to clear)
__device__ __forceinline__ void mma_tf32_z(float (&c)[4], uint32_t a0, uint32_t a1, uint32_t a2,
                                           uint32_t a3, uint32_t b0, uint32_t b1)
{
    asm volatile("mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, "
                 "{%4,%5,%6,%7}, {%8,%9}, {%10,%10,%10,%10};"
                 : "=f"(c[0]), "=f"(c[1]), "=f"(c[2]), "=f"(c[3])
                 : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1), "f"(0.f));
}

static constexpr int TCR = 128;   // rows per CTA (8 warps x 16)
static constexpr int TCJ = 64;    // points per staged tile

// --------------------------------------------------------------------------
// Asynchronous staging.  The point and p tiles are laid out in global memory
// exactly as the compute loop reads them from shared memory -- points as
// duplicated (x, x) pairs, TCJ rows of DS + 2 pairs (Xdup); p split into tf32
// (hi, lo) words, row j = [hi(c), c < NR | pad | lo(c) | pad] of ROW = 2 PS
// words with ROW = 8 mod 32 (conflict-free fragment reads) (Psp) -- both
// padded with zero rows to a multiple of TCJ.  Each tile is then two bulk
// copies (cp.async.bulk, the TMA engine) issued by one thread and completed
// on an mbarrier, double-buffered so that the copies of tile i+1 overlap the
// tensor-core work on tile i.
// --------------------------------------------------------------------------
template <int NB> struct TcRow {
    static constexpr int PS = (NB <= 2) ? 20 : 36;   // hi block + pad, words
    static constexpr int ROW = 2 * PS;               // words per staged p row
};

template <int DS, int NB> struct TcStage {
    static constexpr int PTS = TCJ * (DS + 2) * 8;        // bytes of the point tile
    static constexpr int PB = TCJ * TcRow<NB>::ROW * 4;   // bytes of the p tile
    static constexpr int BYTES = PTS + PB;
};

__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void mbar_init_fence()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}

// global -> shared bulk copy (16-byte aligned addresses, size a multiple of 16)
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes,
                                         uint64_t *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes "
                 "[%0], [%1], %2, [%3];" ::"r"(smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                 " selp.u32 %0, 1, 0, p;\n}"
                 : "=r"(ok)
                 : "r"(smem_addr(bar)), "r"(parity)
                 : "memory");
    return ok != 0;
}

// wait for phase `parity` of the barrier, giving up after 2 s
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity)
{
    uint64_t t0 = 0;
    for (uint32_t spin = 0;; ++spin) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((spin & 63u) == 0) {
            const uint64_t t = globaltimer_ns();
            if (spin == 0) t0 = t;
            else if (t - t0 > 2000000000ull) return false;
        }
    }
}

// Sums sum_{j in [j0, j1)} K(x_i, x_j) p_j for the 16 rows of each warp of a
// 256-thread CTA (rows row0 + warp*16 + {g, g+8}) and the NB groups of 8
// columns of p, with staged tiles read from the prepared Xdup / Psp arrays.
// On return acc[b][.] holds the C-fragment (g,2t) (g,2t+1) (g+8,2t)
// (g+8,2t+1) of column group b.  stage: 2 x TcStage<DS,NB>::BYTES of shared
// memory (16-byte aligned); bars: 2 mbarriers initialised with count 1;
// parity: the phase bits of the two barriers, carried across calls by every
// thread.  Returns false (block-uniformly) when a copy did not complete in
// time; in that case the sums are invalid and the caller reports the error.
template <int DS, int NB, int KER>
__device__ __forceinline__ bool mv32tc_rows_async(const float *__restrict__ Xs, int64_t n,
                                                  const f2_t *__restrict__ Xdup,
                                                  const uint32_t *__restrict__ Psp,
                                                  int64_t row0, int64_t j0, int64_t j1,
                                                  unsigned char *stage, uint64_t *bars,
                                                  uint32_t &parity, float (&acc)[NB][4])
{
    constexpr int ROW = TcRow<NB>::ROW;
    constexpr int PS = TcRow<NB>::PS;
    constexpr int DSP = DS + 2;
    constexpr int SB = TcStage<DS, NB>::BYTES;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = lane >> 2, t = lane & 3;
    const int64_t ia = row0 + warp * 16 + g;
    const int64_t ib = ia + 8;
    f2_t xi[DS];
#pragma unroll
    for (int q = 0; q < DS; ++q)
        xi[q] = f2_pack(ia < n ? Xs[ia * DS + q] : 0.f, ib < n ? Xs[ib * DS + q] : 0.f);
    // running sums and Kahan compensations as packed pairs of the C-fragment
    // registers (0,1) and (2,3): one f32x2 instruction per two elements,
    // rounding identical to the scalar sequence
    f2_t acc2[NB][2], cmp2[TC_KAHAN ? NB : 1][2];
#pragma unroll
    for (int b = 0; b < NB; ++b) acc2[b][0] = acc2[b][1] = 0ull;
#pragma unroll
    for (int b = 0; b < (TC_KAHAN ? NB : 1); ++b) cmp2[b][0] = cmp2[b][1] = 0ull;

    const int ntiles = (int)((j1 - j0 + TCJ - 1) / TCJ);
    auto issue = [&](int it) {
        unsigned char *st = stage + (it & 1) * SB;
        const int64_t j = j0 + (int64_t)it * TCJ;
        uint64_t *bar = bars + (it & 1);
        mbar_expect_tx(bar, (uint32_t)SB);
        bulk_g2s(st, Xdup + j * DSP, (uint32_t)TcStage<DS, NB>::PTS, bar);
        bulk_g2s(st + TcStage<DS, NB>::PTS, Psp + j * ROW, (uint32_t)TcStage<DS, NB>::PB, bar);
    };
    bool ok = true;
    if (threadIdx.x == 0 && ntiles > 0) issue(0);
    int it = 0;
    for (; it < ntiles; ++it) {
        const int b = it & 1;
        if (threadIdx.x == 0 && it + 1 < ntiles) issue(it + 1);
        const bool got = mbar_wait_bounded(bars + b, (parity >> b) & 1u);
        if (!__syncthreads_and(got)) {
            ok = false;      // tile it (and it + 1, if issued) may still be in flight
            break;
        }
        parity ^= 1u << b;
        const f2_t *xsd = reinterpret_cast<const f2_t *>(stage + b * SB);
        const uint32_t *pw = reinterpret_cast<const uint32_t *>(stage + b * SB + TcStage<DS, NB>::PTS);
        float tac[NB][4];
#pragma unroll
        for (int kb = 0; kb < TCJ / 8; ++kb) {
            const f2_t *xa = xsd + (kb * 8 + t) * DSP;
            const f2_t *xb = xsd + (kb * 8 + t + 4) * DSP;
            f2_t ra = 0ull, rb = 0ull;
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
            float r_aa, r_ba, r_ab, r_bb;
            f2_unpack(ra, r_aa, r_ba);
            f2_unpack(rb, r_ab, r_bb);
            uint32_t ah0, al0, ah1, al1, ah2, al2, ah3, al3;
            tf32_split(kernel32_scaled<KER>(r_aa), ah0, al0);
            tf32_split(kernel32_scaled<KER>(r_ba), ah1, al1);
            tf32_split(kernel32_scaled<KER>(r_ab), ah2, al2);
            tf32_split(kernel32_scaled<KER>(r_bb), ah3, al3);
            const uint32_t *p0 = pw + (kb * 8 + t) * ROW + g;
            const uint32_t *p1 = pw + (kb * 8 + t + 4) * ROW + g;
#pragma unroll
            for (int bb = 0; bb < NB; ++bb) {
                const uint32_t bh0 = p0[bb * 8], bh1 = p1[bb * 8];
                const uint32_t bl0 = p0[PS + bb * 8], bl1 = p1[PS + bb * 8];
                // the first product of a fold chunk starts from zero
                if (kb % TC_FOLD == 0) mma_tf32_z(tac[bb], al0, al1, al2, al3, bh0, bh1);
                else mma_tf32(tac[bb], al0, al1, al2, al3, bh0, bh1);
                mma_tf32(tac[bb], ah0, ah1, ah2, ah3, bl0, bl1);
                mma_tf32(tac[bb], ah0, ah1, ah2, ah3, bh0, bh1);
            }
            if ((kb + 1) % TC_FOLD == 0) {
#pragma unroll
                for (int bb = 0; bb < NB; ++bb)
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const f2_t tv = f2_pack(tac[bb][2 * h], tac[bb][2 * h + 1]);
                        if constexpr (TC_KAHAN) {
                            const f2_t y = f2_sub(tv, cmp2[bb][h]);
                            const f2_t s = f2_add(acc2[bb][h], y);
                            cmp2[bb][h] = f2_sub(f2_sub(s, acc2[bb][h]), y);
                            acc2[bb][h] = s;
                        } else {
                            acc2[bb][h] = f2_add(acc2[bb][h], tv);
                        }
                    }
            }
        }
        __syncthreads();   // buffer b is free for the copies of tile it + 2
    }
#pragma unroll
    for (int bb = 0; bb < NB; ++bb) {
        f2_unpack(acc2[bb][0], acc[bb][0], acc[bb][1]);
        f2_unpack(acc2[bb][1], acc[bb][2], acc[bb][3]);
    }
    if (!ok && threadIdx.x == 0) {
        // copies issued but not consumed (tiles it and it + 1): wait for them,
        // again bounded, before the shared memory they write goes out of scope
        for (int k = it; k < ntiles && k <= it + 1; ++k) {
            const int b = k & 1;
            if (mbar_wait_bounded(bars + b, (parity >> b) & 1u)) parity ^= 1u << b;
        }
    }
    return ok;
}

}  // namespace afn
