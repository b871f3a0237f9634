// matvec_umma.cuh -- the FP32 kernel matvec q = K p on the fifth-generation
// tensor cores (tcgen05): kernel values generated on the FP32 pipes straight
// into tensor memory as the A operand, the p tile staged by bulk copies into
// shared memory as the B operand, accumulators in tensor memory.
//
// CTA = 4 UH + 1 warps over 128 rows and one j-chunk:
//   row warps  warp w serves the rows of TMEM lane quarter w % 4, one thread
//              per row, and the share w / 4 of the UH shares of the points and
//              of the columns: for each block of UK points it evaluates
//              K(x_i, x_j) from the staged point tile, splits each value as
//              hi + lo (tf32), stores both into the A buffer of the block
//              (tcgen05.st), and folds its columns of the previous block's
//              accumulator (tcgen05.ld) into an FP32 Kahan sum per column;
//   last warp  one thread issues the bulk copies of the staged tiles and the
//              MMAs: per 8 points D += A_lo B_hi, A_hi B_lo, A_hi B_hi (the
//              three-pass tf32 product, small terms first) with M = 128 rows,
//              N = the right-hand sides; the whole warp owns the TMEM
//              allocation.
// A and D are double-buffered so that the generation of block c + 1, the
// MMAs of block c and the fold of block c - 1 overlap; the staged tiles
// rotate through NST buffers.  Every wait is bounded (the kernel's wait
// limit, 2 s unless afn_set_wait_limit_ns lowered it); a thread that gives up
// raises a CTA-wide abort flag that ends every other wait, and the CTA still
// waits (up to 2 s, whatever the limit) for its copies and MMAs in flight
// before it releases tensor memory and returns.
//
// Operand layouts (PTX ISA, tcgen05): the accumulator and an A operand in
// tensor memory hold row i in lane i, one 32-bit column per element; the B
// tile of one MMA (K = 8 points x N columns, tf32) is K-major without
// swizzle: core matrices of 8 columns x 4 points (128 contiguous bytes, one
// 16-byte row per column), consecutive in the point direction (leading
// byte offset 128) and UJ / 4 core matrices apart in the column direction
// (stride byte offset).
#pragma once

#include "matvec_tc.cuh"

namespace afn {

static constexpr int UR = 128;   // rows per CTA (TMEM lanes)
static constexpr int UJ = 64;    // points per staged tile
static constexpr int UK_DEF = 32;   // points per A block (4 MMA k-steps)
static constexpr int UNST = 3;   // staged tile buffers
static constexpr int UTMEM = 256;   // tensor-memory columns per CTA

// threads per CTA with UH row warps per TMEM lane quarter (they split the
// points of an A block and the accumulator columns of the fold) and one
// issuing warp
__host__ __device__ constexpr int umma_threads(int uh) { return 32 * (4 * uh + 1); }

// The row threads form the squared distance directly, sum_q (x_iq - x_jq)^2,
// two points per f32x2 instruction.
template <int DS, int NR> struct UStage {
    // point tile: pairs (2m + h, q) at float 2m DS + 2q + h
    static constexpr int PTS = UJ * DS * 4;
    static constexpr int PB = UJ * NR * 4;           // one tf32 half of the p tile
    static constexpr int BYTES = PTS + 2 * PB;
};

// ---- tcgen05 wrappers -------------------------------------------------------
__device__ __forceinline__ void tm_fence_before()
{
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tm_fence_after()
{
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// one whole warp: allocate ncols columns, address written to *slot
__device__ __forceinline__ void tm_alloc(uint32_t *slot, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_addr(slot)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tm_dealloc(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
                 : "memory");
}

// D (+)= A B with A in tensor memory, B described in shared memory
__device__ __forceinline__ void umma_tf32(uint32_t dt, uint32_t at, uint64_t bdesc, uint32_t idesc,
                                          uint32_t accumulate)
{
    asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                 " tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n}" ::"r"(dt),
                 "r"(at), "l"(bdesc), "r"(idesc), "r"(accumulate)
                 : "memory");
}

// D (+)= A B with both operands described in shared memory
__device__ __forceinline__ void umma_tf32_ss(uint32_t dt, uint64_t adesc, uint64_t bdesc,
                                             uint32_t idesc, uint32_t accumulate)
{
    asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                 " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(dt),
                 "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
                 : "memory");
}

// arrive once on *bar when every MMA this thread issued so far has completed
__device__ __forceinline__ void umma_commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_addr(bar))
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// 16 columns of this thread's lane: store / load (the load waits for its data)
__device__ __forceinline__ void tm_st16(uint32_t taddr, const uint32_t (&v)[16])
{
    asm volatile("tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, "
                 "%9, %10, %11, %12, %13, %14, %15, %16};" ::"r"(taddr),
                 "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]),
                 "r"(v[7]), "r"(v[8]), "r"(v[9]), "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]),
                 "r"(v[14]), "r"(v[15])
                 : "memory");
}

__device__ __forceinline__ void tm_ld8(uint32_t taddr, uint32_t (&v)[8])
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];\n"
                 "tcgen05.wait::ld.sync.aligned;"
                 : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]),
                   "=r"(v[6]), "=r"(v[7])
                 : "r"(taddr)
                 : "memory");
}

__device__ __forceinline__ void tm_wait_st()
{
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tm_ld16(uint32_t taddr, uint32_t (&v)[16])
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, "
                 "%10, %11, %12, %13, %14, %15}, [%16];\n"
                 "tcgen05.wait::ld.sync.aligned;"
                 : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]),
                   "=r"(v[6]), "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]),
                   "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
                 : "r"(taddr)
                 : "memory");
}

// shared-memory matrix descriptor: no swizzle, byte offsets lbo (point
// direction) and sbo (column direction), descriptor version 1
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// instruction descriptor: D f32, A and B tf32 (both K-major), M x N
__host__ __device__ constexpr uint32_t umma_idesc_tf32(int M, int N)
{
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}

// bounded wait that also ends when another thread of the CTA has given up;
// limit_ns is the kernel's wait limit (afn_set_wait_limit_ns, default 2 s)
__device__ __forceinline__ bool mbar_wait_abort(uint64_t *bar, uint32_t parity, volatile int *abort,
                                                uint64_t limit_ns)
{
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = globaltimer_ns();
    for (;;) {
        if (mbar_try_wait(bar, parity)) return true;
        if (*abort) return false;
        if (globaltimer_ns() - t0 > limit_ns) {
            *abort = 1;
            return false;
        }
    }
}

// warp-uniform variant (all lanes wait, all take the same branch)
__device__ __forceinline__ bool mbar_wait_abort_warp(uint64_t *bar, uint32_t parity,
                                                     volatile int *abort, uint64_t limit_ns)
{
    const bool got = mbar_wait_abort(bar, parity, abort, limit_ns);
    return __all_sync(0xffffffffu, got);
}

// Kahan fold of C accumulator columns (packed pairs) into acc / cmp
template <int C>
__device__ __forceinline__ void umma_fold(const uint32_t (&v)[C], f2_t *acc, f2_t *cmp)
{
#pragma unroll
    for (int h = 0; h < C / 2; ++h) {
        const f2_t tv = f2_pack(__uint_as_float(v[2 * h]), __uint_as_float(v[2 * h + 1]));
        if constexpr (TC_KAHAN) {
            const f2_t y = f2_sub(tv, cmp[h]);
            const f2_t s = f2_add(acc[h], y);
            cmp[h] = f2_sub(f2_sub(s, acc[h]), y);
            acc[h] = s;
        } else {
            acc[h] = f2_add(acc[h], tv);
        }
    }
}

// Sums over the stages [s0, s1) of the prepared arrays:
//   Xpr: per stage of UJ points the point tile of UStage (zero rows up to a
//        multiple of UJ);
//   Pk:  per stage of UJ points, the tf32 hi then lo halves of p in the
//        K-major core-matrix layout above (word (c/8)(UJ/4)32 + (jj/4)32 +
//        (c%8)4 + jj%4 for point jj of the stage and column c).
// Row sums of rows [row0, row0 + 128) leave through part (column-major per
// chunk, leading dimension n).
// two CTAs per SM (their TMEM allocations fit together) when the registers allow
__host__ __device__ constexpr int umma_min_blocks(int uh) { return umma_threads(uh) * 2 * 168 <= 65536 ? 2 : 1; }

template <int DS, int NB, int KER, int UH>
__global__ void __launch_bounds__(umma_threads(UH), umma_min_blocks(UH))
    matvec32u_kernel(const float *__restrict__ Xs, int64_t n, const float *__restrict__ Xpr,
                     const uint32_t *__restrict__ Pk, float *__restrict__ part, int64_t chunk_st,
                     int64_t nstage, int *__restrict__ err, uint64_t wait_ns)
{
    constexpr int NR = NB * 8;
    constexpr int UPW = 4 * UH;                  // row warps
    constexpr int UK = UK_DEF;
    constexpr int SB = UStage<DS, NR>::BYTES;
    constexpr int PTS = UStage<DS, NR>::PTS;
    constexpr int BPS = UJ / UK;                 // A blocks per staged tile
    constexpr uint32_t IDESC = umma_idesc_tf32(UR, NR);
    // tensor-memory columns: A buffers (hi | lo) then the accumulators
    constexpr uint32_t COL_A = 0, COL_D = 4 * UK;
    static_assert(COL_D + 2 * NR <= UTMEM, "tensor memory");
    static_assert(UJ % UK == 0 && UK % (16 * UH) == 0 && NR % 16 == 0, "tile shape");
    constexpr int FC = NR / UH;                  // accumulator columns folded per thread
    static_assert(FC % 8 == 0, "fold width");

    extern __shared__ __align__(128) unsigned char usm[];
    __shared__ __align__(8) uint64_t full[UNST], empty[UNST], afull[2], bdone[2], dempty[2], fin;
    __shared__ uint32_t tbase_slot;
    __shared__ int abort_flag;
    volatile int *abort = &abort_flag;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t row0 = (int64_t)blockIdx.x * UR;
    const int64_t s0 = (int64_t)blockIdx.y * chunk_st;
    const int64_t s1 = min(nstage, s0 + chunk_st);
    const int nst = (int)(s1 - s0);
    const int nblk = nst * BPS;

    if (threadIdx.x == 0) {
        for (int b = 0; b < UNST; ++b) {
            mbar_init(&full[b], 1);
            mbar_init(&empty[b], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&afull[b], UPW);
            mbar_init(&bdone[b], 1);
            mbar_init(&dempty[b], UPW);
        }
        mbar_init(&fin, 1);
        abort_flag = 0;
        mbar_init_fence();
    }
    if (warp == UPW) tm_alloc(&tbase_slot, UTMEM);
    tm_fence_before();
    __syncthreads();
    tm_fence_after();
    const uint32_t tbase = tbase_slot;

    if (warp == UPW) {
        // ------------------------------------------------ copies and MMAs --
        if (lane == 0) {
            int issued = 0;     // staged tiles whose copies were issued
            int observed = 0;   // staged tiles whose completion was observed here
            auto issue = [&](int s) {
                unsigned char *st = usm + (s % UNST) * SB;
                uint64_t *bar = &full[s % UNST];
                mbar_expect_tx(bar, (uint32_t)SB);
                bulk_g2s(st, Xpr + (s0 + s) * (PTS / 4), (uint32_t)PTS, bar);
                bulk_g2s(st + PTS, Pk + (s0 + s) * (int64_t)(2 * UJ * NR),
                         (uint32_t)(2 * UStage<DS, NR>::PB), bar);
            };
            for (; issued < nst && issued < UNST; ++issued) issue(issued);
            const uint32_t base_s = smem_addr(usm);
            for (int c = 0; c < nblk && !*abort; ++c) {
                const int b = c & 1;
                const int s = c / BPS, sb = s % UNST;
                if (c % BPS == 0) {
                    if (!mbar_wait_abort(&full[sb], (uint32_t)(s / UNST) & 1u, abort, wait_ns)) break;
                    observed = s + 1;
                }
                if (!mbar_wait_abort(&afull[b], (uint32_t)(c >> 1) & 1u, abort, wait_ns)) break;
                if (c >= 2 && !mbar_wait_abort(&dempty[b], (uint32_t)((c - 2) >> 1) & 1u, abort, wait_ns))
                    break;
                tm_fence_after();
                const uint32_t phi = base_s + sb * SB + PTS;
                const uint32_t plo = phi + UStage<DS, NR>::PB;
                const uint32_t a_hi = tbase + COL_A + b * 2 * UK, a_lo = a_hi + UK;
                const uint32_t dcol = tbase + COL_D + b * NR;
#pragma unroll
                for (int q = 0; q < UK / 8; ++q) {
                    // core-matrix column of this k-step within the stage
                    const uint32_t off = (uint32_t)(((c % BPS) * (UK / 4) + 2 * q) * 128);
                    const uint64_t dh = umma_desc(phi + off, 128, (UJ / 4) * 128);
                    const uint64_t dl = umma_desc(plo + off, 128, (UJ / 4) * 128);
                    umma_tf32(dcol, a_lo + 8 * q, dh, IDESC, q > 0);
                    umma_tf32(dcol, a_hi + 8 * q, dl, IDESC, 1);
                    umma_tf32(dcol, a_hi + 8 * q, dh, IDESC, 1);
                }
                umma_commit(&bdone[b]);
                if (c % BPS == BPS - 1) {
                    umma_commit(&empty[sb]);
                    if (issued < nst) {
                        // refill this buffer once its MMAs are done
                        if (!mbar_wait_abort(&empty[sb], (uint32_t)(s / UNST) & 1u, abort, wait_ns)) break;
                        issue(issued++);
                    }
                }
            }
            // drain (bounded): every MMA issued so far, then every copy whose
            // completion this thread has not observed
            umma_commit(&fin);
            mbar_wait_bounded(&fin, 0);
            for (int s = observed; s < issued; ++s)
                mbar_wait_bounded(&full[s % UNST], (uint32_t)(s / UNST) & 1u);
        }
        __syncwarp();
    } else {
        // ------------------------------------------------ rows -------------
        const int quarter = warp & 3, hf = warp >> 2;
        const int64_t i = row0 + quarter * 32 + lane;
        f2_t xi2[DS];
#pragma unroll
        for (int q = 0; q < DS; ++q) {
            const float v = i < n ? Xs[i * DS + q] : 0.f;
            xi2[q] = f2_pack(v, v);
        }
        f2_t acc[FC / 2], cmp[FC / 2];
#pragma unroll
        for (int h = 0; h < FC / 2; ++h) acc[h] = cmp[h] = 0ull;
        const uint32_t lane_off = (uint32_t)(quarter * 32) << 16;
        auto fold = [&](int c) -> bool {
            if (!mbar_wait_abort_warp(&bdone[c & 1], (uint32_t)(c >> 1) & 1u, abort, wait_ns)) return false;
            tm_fence_after();
            const uint32_t dcol = tbase + lane_off + COL_D + (c & 1) * NR + hf * FC;
            if constexpr (FC % 16 == 0) {
#pragma unroll
                for (int h = 0; h < FC / 16; ++h) {
                    uint32_t v[16];
                    tm_ld16(dcol + 16 * h, v);
                    umma_fold<16>(v, acc + 8 * h, cmp + 8 * h);
                }
            } else {
#pragma unroll
                for (int h = 0; h < FC / 8; ++h) {
                    uint32_t v[8];
                    tm_ld8(dcol + 8 * h, v);
                    umma_fold<8>(v, acc + 4 * h, cmp + 4 * h);
                }
            }
            tm_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&dempty[c & 1]);
            return true;
        };
        bool ok = true;
        for (int c = 0; c < nblk && ok; ++c) {
            const int b = c & 1;
            const int s = c / BPS, sb = s % UNST;
            if (c % BPS == 0 && !mbar_wait_abort_warp(&full[sb], (uint32_t)(s / UNST) & 1u, abort, wait_ns)) {
                ok = false;
                break;
            }
            // A buffer b was last read by the MMAs of block c - 2, whose
            // completion the fold of block c - 2 (previous iteration) awaited.
            // This warp's points: UK / UH of the block, in groups of 16.
            const unsigned char *tile = usm + sb * SB;
            const int jb = (c % BPS) * UK + hf * (UK / UH);   // first point of this warp
            const uint32_t a_hi = tbase + lane_off + COL_A + b * 2 * UK + hf * (UK / UH);
            const uint32_t a_lo = a_hi + UK;
#pragma unroll
            for (int g16 = 0; g16 < UK / (16 * UH); ++g16) {
                uint32_t vh[16], vl[16];
                const int j16 = jb + 16 * g16;
                const f2_t *xp = reinterpret_cast<const f2_t *>(tile) + j16 / 2 * DS;
#pragma unroll
                for (int m = 0; m < 8; ++m) {
                    const f2_t *pp = xp + m * DS;
                    f2_t r = 0ull;
#pragma unroll
                    for (int q = 0; q < DS; q += 2) {
                        const ulonglong2 v = *reinterpret_cast<const ulonglong2 *>(pp + q);
                        f2_t u = f2_sub(xi2[q], v.x);
                        r = f2_fma(u, u, r);
                        u = f2_sub(xi2[q + 1], v.y);
                        r = f2_fma(u, u, r);
                    }
                    float r0, r1;
                    f2_unpack(r, r0, r1);
                    tf32_split(kernel32_scaled<KER>(r0), vh[2 * m], vl[2 * m]);
                    tf32_split(kernel32_scaled<KER>(r1), vh[2 * m + 1], vl[2 * m + 1]);
                }
                tm_st16(a_hi + 16 * g16, vh);
                tm_st16(a_lo + 16 * g16, vl);
            }
            tm_wait_st();
            tm_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&afull[b]);
            if (c >= 1 && !fold(c - 1)) ok = false;
        }
        if (ok && nblk > 0 && !fold(nblk - 1)) ok = false;
        if (ok && i < n) {
#pragma unroll
            for (int h = 0; h < FC / 2; ++h) {
                float a0, a1;
                f2_unpack(acc[h], a0, a1);
                const int col = hf * FC + 2 * h;
                part[((int64_t)blockIdx.y * NR + col) * n + i] = a0;
                part[((int64_t)blockIdx.y * NR + col + 1) * n + i] = a1;
            }
        }
        tm_fence_before();
    }
    __syncthreads();
    if (warp == UPW) {
        tm_fence_after();
        tm_dealloc(tbase, UTMEM);
    }
    if (threadIdx.x == 0 && *abort) atomicExch(err, DEV_TIMEOUT);
}

}  // namespace afn
