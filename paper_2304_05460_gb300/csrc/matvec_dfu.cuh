// matvec_dfu.cuh -- the FP64-accurate kernel matvec q = K p with the
// contraction on the fifth-generation tensor cores.
//
// The kernel values are formed in double-float on the FP32 pipes exactly as
// in the CUDA-core double-float matvec (matvec_df.cuh); only the sum over j
// moves to tcgen05.  It is made exact there by splitting both operands into
// fixed-point base-256 digits (the error-free splitting of Ozaki, Ogita, Oishi
// and Rump, "Error-free transformations of matrix multiplication by using
// fast routines of matrix multiplication", Numer. Algorithms 59, 2012, in its
// fixed-point form):
//
//   K_ij      = sum_{s<8} a_s(i,j) 2^(-7-8s),        0 <= K_ij <= 1,
//   p_jc      = 2^(E_c) sum_{t<8} b_t(j,c) 2^(-7-8t), 2^(E_c) > max_j |p_jc|,
//
// with integer digits |a_s| <= 192 and |b_t| <= 128, all exact in BF16.  For
// a block of 32 points the products a_s b_t are integers below 2^15, and
//   D_q(i,c) = sum_{s+t=q} sum_j a_s(i,j) b_t(j,c),   q = 0..7,
// stays below 8 * 32 * 192 * 128 < 2^23, so the FP32 accumulation of the BF16
// MMAs forms every D_q exactly.  The block's contribution to q_ic is
// 2^(E_c - 14) sum_q D_q 2^(-8q); the terms dropped (s + t >= 8) and the
// digits cut off are below 2^-61 max|p_c| per product term.
//
// One MMA per (digit s, k-step) forms all D_q with q >= s at once: its B
// operand is the digit tile [b_0 | b_1 | ... | b_(7-s)] (N = 32 (8 - s)
// columns) and its accumulator starts at the TMEM column of D_s, so digit t
// of p lands in D_(s+t).  The fold adds, per block and column, the exact
// integer H = D_0 2^16 + D_1 2^8 + D_2 into an int64 and the rest
// (D_3 2^-8 + ... + D_7 2^-40, relative weight 2^-24) into an FP32 Kahan sum;
// the result is 2^(E_c - 30) (H + L).
//
// CTA = 17 warps over 128 rows and one j-chunk:
//   row warps  warp w serves TMEM lane quarter w % 4 and the 8 points w / 4
//              of each block: it evaluates their kernel values, writes their
//              digits into the A tile of the block in shared memory (the
//              K-major core-matrix layout of the MMA), and folds its 8
//              columns of the previous block's accumulator;
//   last warp  one thread issues the bulk copies of the staged tiles (points
//              and p digits, one stage per block) and the 16 MMAs of a
//              block (8 digits x 2 k-steps of 16 points), M = 128.
// The A tile is double-buffered; the accumulator (256 TMEM columns) is
// single: the MMAs of block c wait for the fold of block c - 1, which is
// short next to the evaluation of block c + 1 that runs meanwhile.  Every
// wait is bounded (the kernel's wait limit) with a CTA-wide abort flag and a
// bounded drain, as in the FP32 tcgen05 matvec.
#pragma once

#include "gemm_bf16.cuh"
#include "matvec_df.cuh"

namespace afn {

static constexpr int DU_J = 32;      // points per block (= per staged tile)
static constexpr int DU_DIG = 8;     // digits of K and of p
static constexpr int DU_NR = 32;     // columns of p per launch
static constexpr int DU_NST = 4;     // staged tile buffers
static constexpr int DU_UH = 4;      // row warps per TMEM lane quarter
static constexpr int DU_THREADS = 32 * (4 * DU_UH + 1);
static constexpr int DU_TMEM = DU_DIG * DU_NR;               // 256 accumulator columns
static constexpr int DU_ATILE = UR * DU_J * 2;               // one digit of A (8 KB)
static constexpr int DU_ABUF = DU_DIG * DU_ATILE;            // all digits of a block
static constexpr int DU_PDIG = DU_J * DU_DIG * DU_NR * 2;    // digit tile of p (16 KB)

template <int DS> struct DuStage {
    static constexpr int PTS = DU_J * DS * 8;                // double-float points
    static constexpr int BYTES = PTS + DU_PDIG;
    static constexpr int SMEM = 2 * DU_ABUF + DU_NST * BYTES;
};

// element of (column n', point kk) in a DU_J-point digit tile of p, and of
// (row r, point kk) in a digit tile of A: K-major core matrices of 8 rows x
// 8 points (16-byte rows), DU_J / 8 core matrices along K
__host__ __device__ inline int64_t du_tile_elem(int r, int kk)
{
    return (int64_t)((r / 8) * (DU_J / 8) + kk / 8) * 64 + (r % 8) * 8 + (kk % 8);
}

__device__ __forceinline__ void fence_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// nearest multiple of g = 2^(-7-8s) to r, with c = 1.5 * 2^23 * g (|r| < 2^22 g),
// two values
__device__ __forceinline__ f2_t du_round2(f2_t r, float c)
{
    return f2_sub(f2_add(r, f2_splat(c)), f2_splat(c));
}

// the eight base-256 digits of two double-float kernel values 0 <= v <= 1:
// v = sum_s d[s] 2^(-7-8s) up to 2^-64; the low float is merged into the
// remainder twice (after digits 2 and 5), where it can first reach a digit
__device__ __forceinline__ void du_digits2(dfl2 v, f2_t (&d)[DU_DIG])
{
    f2_t r = v.h, rl = v.l, a;
    a = du_round2(r, 0x1.8p16f);  r = f2_sub(r, a); d[0] = f2_mul(a, f2_splat(0x1p7f));
    a = du_round2(r, 0x1.8p8f);   r = f2_sub(r, a); d[1] = f2_mul(a, f2_splat(0x1p15f));
    a = du_round2(r, 0x1.8p0f);   r = f2_sub(r, a); d[2] = f2_mul(a, f2_splat(0x1p23f));
    two_sum2(r, rl, r, rl);
    a = du_round2(r, 0x1.8p-8f);  r = f2_sub(r, a); d[3] = f2_mul(a, f2_splat(0x1p31f));
    a = du_round2(r, 0x1.8p-16f); r = f2_sub(r, a); d[4] = f2_mul(a, f2_splat(0x1p39f));
    a = du_round2(r, 0x1.8p-24f); r = f2_sub(r, a); d[5] = f2_mul(a, f2_splat(0x1p47f));
    two_sum2(r, rl, r, rl);
    a = du_round2(r, 0x1.8p-32f); r = f2_sub(r, a); d[6] = f2_mul(a, f2_splat(0x1p55f));
    a = du_round2(f2_add(r, rl), 0x1.8p-40f);       d[7] = f2_mul(a, f2_splat(0x1p63f));
}

__device__ __forceinline__ uint32_t du_pack(float lo, float hi)
{
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);   // .x (low half) = lo
    return *reinterpret_cast<const uint32_t *>(&v);
}

// exact integer value of an FP32 accumulator entry (|x| < 2^22)
__device__ __forceinline__ int du_int(float x)
{
    return __float_as_int(__fadd_rn(x, 0x1.8p23f)) - 0x4B400000;
}

// Row sums over the stages [s0, s1) of the prepared arrays:
//   Xs:  the double-float points of the rows (n x DS);
//   Xpr: per stage the DU_J staged points (n padded with zero points) as
//        packed pairs: points 2m, 2m + 1 and dimension q at float4 m DS + q =
//        {h(2m), h(2m + 1), l(2m), l(2m + 1)};
//   Pd:  per stage the digit tile of p (column n' = 32 t + c holds digit t of
//        column c, du_tile_elem layout), zero beyond n and beyond nc columns;
//   pexp: E_c per column.
// part: column-major per chunk, leading dimension n, nc columns per chunk.
template <int DS, int KER>
__global__ void __launch_bounds__(DU_THREADS, 1)
    matvecdfu_kernel(const float2 *__restrict__ Xs, int64_t n, const float2 *__restrict__ Xpr,
                     const __nv_bfloat16 *__restrict__ Pd, const int *__restrict__ pexp,
                     double *__restrict__ part, int nc, int64_t chunk_st, int64_t nstage,
                     int *__restrict__ err, uint64_t wait_ns)
{
    constexpr int PTS = DuStage<DS>::PTS;
    constexpr int SB = DuStage<DS>::BYTES;
    constexpr int UPW = 4 * DU_UH;               // row warps
    constexpr int FC = DU_NR / DU_UH;            // accumulator columns folded per thread
    static_assert(FC == 8 && DU_J == 8 * DU_UH, "tile shape");

    extern __shared__ __align__(128) unsigned char dusm[];
    __shared__ __align__(8) uint64_t full[DU_NST], empty[DU_NST], afull[2], bdone, dempty, fin;
    __shared__ uint32_t tbase_slot;
    __shared__ int abort_flag;
    __shared__ DfExpTable T;
    volatile int *abort = &abort_flag;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t row0 = (int64_t)blockIdx.x * UR;
    const int64_t s0 = (int64_t)blockIdx.y * chunk_st;
    const int64_t s1 = min(nstage, s0 + chunk_st);
    const int nblk = (int)(s1 - s0);
    unsigned char *abuf = dusm;                          // 2 x DU_ABUF
    unsigned char *stages = dusm + 2 * DU_ABUF;          // DU_NST x SB

    df_table_init(T);
    if (threadIdx.x == 0) {
        for (int b = 0; b < DU_NST; ++b) {
            mbar_init(&full[b], 1);
            mbar_init(&empty[b], 1);
        }
        mbar_init(&afull[0], UPW);
        mbar_init(&afull[1], UPW);
        mbar_init(&bdone, 1);
        mbar_init(&dempty, UPW);
        mbar_init(&fin, 1);
        abort_flag = 0;
        mbar_init_fence();
    }
    if (warp == UPW) tm_alloc(&tbase_slot, DU_TMEM);
    tm_fence_before();
    __syncthreads();
    tm_fence_after();
    const uint32_t tbase = tbase_slot;

    if (warp == UPW) {
        // ------------------------------------------------ copies and MMAs --
        if (lane == 0) {
            int issued = 0, observed = 0;
            auto issue = [&](int st) {
                unsigned char *dst = stages + (st % DU_NST) * SB;
                uint64_t *bar = &full[st % DU_NST];
                mbar_expect_tx(bar, (uint32_t)SB);
                bulk_g2s(dst, Xpr + (s0 + st) * (int64_t)(DU_J * DS), (uint32_t)PTS, bar);
                bulk_g2s(dst + PTS, Pd + (s0 + st) * (int64_t)(DU_J * DU_DIG * DU_NR),
                         (uint32_t)DU_PDIG, bar);
            };
            for (; issued < nblk && issued < DU_NST; ++issued) issue(issued);
            const uint32_t a_s = smem_addr(abuf), st_s = smem_addr(stages);
            for (int c = 0; c < nblk && !*abort; ++c) {
                const int sb = c % DU_NST;
                if (!mbar_wait_abort(&full[sb], (uint32_t)(c / DU_NST) & 1u, abort, wait_ns)) break;
                observed = c + 1;
                if (!mbar_wait_abort(&afull[c & 1], (uint32_t)(c >> 1) & 1u, abort, wait_ns)) break;
                if (c >= 1 && !mbar_wait_abort(&dempty, (uint32_t)(c - 1) & 1u, abort, wait_ns)) break;
                tm_fence_after();
                const uint32_t a0 = a_s + (uint32_t)((c & 1) * DU_ABUF);
                const uint32_t p0 = st_s + (uint32_t)(sb * SB + PTS);
#pragma unroll
                for (int k16 = 0; k16 < DU_J / 16; ++k16) {
                    const uint64_t db = umma_desc(p0 + k16 * 256, 128, (DU_J / 8) * 128);
#pragma unroll
                    for (int s = 0; s < DU_DIG; ++s) {
                        const uint64_t da = umma_desc(a0 + s * DU_ATILE + k16 * 256, 128, (DU_J / 8) * 128);
                        umma_bf16_ss(tbase + (uint32_t)(s * DU_NR), da, db,
                                     umma_idesc_bf16(UR, (DU_DIG - s) * DU_NR),
                                     (k16 > 0 || s > 0) ? 1u : 0u);
                    }
                }
                umma_commit(&bdone);
                umma_commit(&empty[sb]);
                // refill the buffer of the previous block, whose MMAs were issued a block earlier
                if (c >= 1 && issued < nblk) {
                    const int cp = c - 1;
                    if (!mbar_wait_abort(&empty[cp % DU_NST], (uint32_t)(cp / DU_NST) & 1u, abort, wait_ns))
                        break;
                    issue(issued++);
                }
            }
            // drain (bounded): every MMA issued so far, then every copy whose
            // completion this thread has not observed
            umma_commit(&fin);
            mbar_wait_bounded(&fin, 0);
            for (int st = observed; st < issued; ++st)
                mbar_wait_bounded(&full[st % DU_NST], (uint32_t)(st / DU_NST) & 1u);
        }
        __syncwarp();
    } else {
        // ------------------------------------------------ rows -------------
        const int quarter = warp & 3, hf = warp >> 2;
        const int r = quarter * 32 + lane;               // row within the tile = TMEM lane
        const int64_t i = row0 + r;
        dfl xi[DS];
#pragma unroll
        for (int q = 0; q < DS; ++q) {
            const float2 v = i < n ? Xs[i * DS + q] : make_float2(0.f, 0.f);
            xi[q] = dfl{v.x, v.y};
        }
        long long hacc[FC];
        float lsum[FC], lcmp[FC];
#pragma unroll
        for (int e = 0; e < FC; ++e) {
            hacc[e] = 0;
            lsum[e] = lcmp[e] = 0.f;
        }
        const uint32_t lane_off = (uint32_t)(quarter * 32) << 16;
        // this thread's 16-byte row of its core matrix in each digit tile of A
        const int aoff = (int)du_tile_elem(r, hf * 8) * 2;
        auto fold = [&](int c) -> bool {
            if (!mbar_wait_abort_warp(&bdone, (uint32_t)c & 1u, abort, wait_ns)) return false;
            tm_fence_after();
            const uint32_t dcol = tbase + lane_off + (uint32_t)(hf * FC);
            uint32_t v0[8], v1[8], v2[8];
            tm_ld8(dcol + 0 * DU_NR, v0);
            tm_ld8(dcol + 1 * DU_NR, v1);
            tm_ld8(dcol + 2 * DU_NR, v2);
#pragma unroll
            for (int e = 0; e < FC; ++e) {
                const int i0 = du_int(__uint_as_float(v0[e]));
                const int t12 = du_int(__uint_as_float(v1[e])) * 256 + du_int(__uint_as_float(v2[e]));
                hacc[e] += (long long)i0 * 65536 + (long long)t12;
            }
            float f[8];
            {
                uint32_t v[8];
                tm_ld8(dcol + 7 * DU_NR, v);
#pragma unroll
                for (int e = 0; e < FC; ++e) f[e] = __uint_as_float(v[e]) * 0x1p-40f;
#pragma unroll
                for (int q = 6; q >= 3; --q) {
                    tm_ld8(dcol + q * DU_NR, v);
                    const float w = q == 6 ? 0x1p-32f : q == 5 ? 0x1p-24f : q == 4 ? 0x1p-16f : 0x1p-8f;
#pragma unroll
                    for (int e = 0; e < FC; ++e) f[e] = __fmaf_rn(__uint_as_float(v[e]), w, f[e]);
                }
            }
#pragma unroll
            for (int e = 0; e < FC; ++e) {
                const float y = __fsub_rn(f[e], lcmp[e]);
                const float t = __fadd_rn(lsum[e], y);
                lcmp[e] = __fsub_rn(__fsub_rn(t, lsum[e]), y);
                lsum[e] = t;
            }
            tm_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&dempty);
            return true;
        };
        bool ok = true;
        for (int c = 0; c < nblk && ok; ++c) {
            const int sb = c % DU_NST;
            if (!mbar_wait_abort_warp(&full[sb], (uint32_t)(c / DU_NST) & 1u, abort, wait_ns)) {
                ok = false;
                break;
            }
            // A buffer c & 1 was last read by the MMAs of block c - 2, whose
            // completion the fold of block c - 2 (previous iteration) awaited
            const float4 *pts = reinterpret_cast<const float4 *>(stages + sb * SB);
            unsigned char *ab = abuf + (c & 1) * DU_ABUF + aoff;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                uint32_t w[DU_DIG][2];
#pragma unroll
                for (int m2 = 0; m2 < 2; ++m2) {
                    // points jj and jj + 1 together (packed pairs of the staged tile)
                    f2_t d2[DU_DIG];
                    const int jj = hf * 8 + h * 4 + m2 * 2;
                    du_digits2(df_kernel2<KER>(df_dist2_2<DS>(xi, pts + (jj / 2) * DS), T), d2);
#pragma unroll
                    for (int s = 0; s < DU_DIG; ++s) {
                        float a0, a1;
                        f2_unpack(d2[s], a0, a1);
                        w[s][m2] = du_pack(a0, a1);
                    }
                }
#pragma unroll
                for (int s = 0; s < DU_DIG; ++s)
                    *reinterpret_cast<uint2 *>(ab + s * DU_ATILE + h * 8) = make_uint2(w[s][0], w[s][1]);
            }
            fence_async_smem();
            __syncwarp();
            if (lane == 0) mbar_arrive(&afull[c & 1]);
            if (c >= 1 && !fold(c - 1)) ok = false;
        }
        if (ok && nblk > 0 && !fold(nblk - 1)) ok = false;
        if (ok && i < n) {
#pragma unroll
            for (int e = 0; e < FC; ++e) {
                const int col = hf * FC + e;
                if (col < nc) {
                    const double v = (double)hacc[e] + ((double)lsum[e] - (double)lcmp[e]);
                    part[((int64_t)blockIdx.y * nc + col) * n + i] = ldexp(v, pexp[col] - 30);
                }
            }
        }
        tm_fence_before();
    }
    __syncthreads();
    if (warp == UPW) {
        tm_fence_after();
        tm_dealloc(tbase, DU_TMEM);
    }
    if (threadIdx.x == 0 && *abort) atomicExch(err, DEV_TIMEOUT);
}

}  // namespace afn
