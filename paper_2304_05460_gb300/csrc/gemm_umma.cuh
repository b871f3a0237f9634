// gemm_umma.cuh -- the two W products of the FP32 preconditioner apply on the
// fifth-generation tensor cores (tcgen05):
//   t = r2 - W^T z'   (rows i of W^T, K = the k landmarks)
//   u = z' - W s2     (rows p of W,   K = the n_r remaining points)
// Each operand matrix is stored once per build in a tiled image (row tile of
// 128 x stage of GKU K-elements, the K-major core-matrix layout of the MMA),
// so a stage is one contiguous bulk copy.  The product keeps FP32 accuracy
// with the three-pass tf32 split of both operands: the 128 x GKU tile is
// split into hi / lo words in shared memory by the row warps after it lands,
// the vector block arrives already split, and
//   D += A_lo B_hi + A_hi B_lo + A_hi B_hi
// accumulates in tensor memory; the row warps fold D into FP32 Kahan sums
// after every stage.
//
// CTA = 9 warps: warps 0-7 split the staged tile (256 threads over 4096
// words) and fold the accumulator (warp w: TMEM lane quarter w % 4, columns
// half w / 4), warp 8 issues the copies and the MMAs and owns the TMEM
// allocation.  Stages rotate through GNST buffers; the accumulator is
// double-buffered.  Every wait is bounded (the wait limit, 2 s by default) with a CTA-wide
// abort flag; the drain after an abort waits up to 2 s for copies in flight.
#pragma once

#include "matvec_umma.cuh"

namespace afn {

static constexpr int GKU = 32;      // K-elements per stage (4 MMA k-steps)
static constexpr int GNST = 4;      // stage buffers
static constexpr int GUT = 288;     // threads: 8 split/fold warps + 1 issuing warp
static constexpr int GU_TMEM = 64;  // two accumulators of up to 32 columns

template <int NR> struct GStage {
    static constexpr int AB = UR * GKU * 4;      // one operand tile (raw, then hi) bytes
    static constexpr int BB = GKU * NR * 4;      // one tf32 half of the vector block
    static constexpr int BYTES = 2 * AB + 2 * BB;
};

// part[(y NR + c) M + i] = sum over the CTA's stages of A[i, :] B[:, c] for the
// 128 rows of row tile blockIdx.x; Atl: the tiled operand, row tiles of
// nks stages each (4096 words a stage); Bk: the split vector block, per stage
// the hi then lo halves in the K-major core-matrix layout (word
// (c/8)(GKU/4)32 + (kk/4)32 + (c%8)4 + kk%4).
template <int NB>
__global__ void __launch_bounds__(GUT, 1)
    gemm32u_kernel(const float *__restrict__ Atl, int64_t M, int64_t nks,
                   const uint32_t *__restrict__ Bk, float *__restrict__ part, int64_t chunk_st,
                   int *__restrict__ err, uint64_t wait_ns)
{
    constexpr int NR = NB * 8;
    constexpr int AB = GStage<NR>::AB, BB = GStage<NR>::BB, SB = GStage<NR>::BYTES;
    constexpr uint32_t IDESC = umma_idesc_tf32(UR, NR);
    constexpr int FC = NR / 2;   // columns folded per thread
    static_assert(NR % 16 == 0 && FC % 8 == 0, "shape");

    extern __shared__ __align__(128) unsigned char gsm[];
    __shared__ __align__(8) uint64_t full[GNST], empty[GNST], split[GNST], bdone[2], dempty[2], fin;
    __shared__ uint32_t tbase_slot;
    __shared__ int abort_flag;
    volatile int *abort = &abort_flag;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t rt = blockIdx.x;
    const int64_t s0 = (int64_t)blockIdx.y * chunk_st;
    const int nst = (int)(min(nks, s0 + chunk_st) - s0);

    if (threadIdx.x == 0) {
        for (int b = 0; b < GNST; ++b) {
            mbar_init(&full[b], 1);
            mbar_init(&empty[b], 1);
            mbar_init(&split[b], 8);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&bdone[b], 1);
            mbar_init(&dempty[b], 8);
        }
        mbar_init(&fin, 1);
        abort_flag = 0;
        mbar_init_fence();
    }
    if (warp == 8) tm_alloc(&tbase_slot, GU_TMEM);
    tm_fence_before();
    __syncthreads();
    tm_fence_after();
    const uint32_t tbase = tbase_slot;

    if (warp == 8) {
        if (lane == 0) {
            int issued = 0, observed = 0;
            auto issue = [&](int s) {
                unsigned char *st = gsm + (s % GNST) * SB;
                uint64_t *bar = &full[s % GNST];
                mbar_expect_tx(bar, (uint32_t)(AB + 2 * BB));
                bulk_g2s(st, Atl + (rt * nks + s0 + s) * (int64_t)(UR * GKU), (uint32_t)AB, bar);
                bulk_g2s(st + 2 * AB, Bk + (s0 + s) * (int64_t)(2 * GKU * NR), (uint32_t)(2 * BB), bar);
            };
            for (; issued < nst && issued < GNST; ++issued) issue(issued);
            const uint32_t base_s = smem_addr(gsm);
            for (int s = 0; s < nst && !*abort; ++s) {
                const int sb = s % GNST, b = s & 1;
                if (!mbar_wait_abort(&full[sb], (uint32_t)(s / GNST) & 1u, abort, wait_ns)) break;
                observed = s + 1;
                if (!mbar_wait_abort(&split[sb], (uint32_t)(s / GNST) & 1u, abort, wait_ns)) break;
                if (s >= 2 && !mbar_wait_abort(&dempty[b], (uint32_t)((s - 2) >> 1) & 1u, abort, wait_ns)) break;
                tm_fence_after();
                const uint32_t ahi = base_s + sb * SB, alo = ahi + AB;
                const uint32_t bhi = ahi + 2 * AB, blo = bhi + BB;
                const uint32_t dcol = tbase + b * NR;
#pragma unroll
                for (int q = 0; q < GKU / 8; ++q) {
                    const uint32_t off = (uint32_t)(2 * q * 128);
                    const uint64_t dah = umma_desc(ahi + off, 128, (GKU / 4) * 128);
                    const uint64_t dal = umma_desc(alo + off, 128, (GKU / 4) * 128);
                    const uint64_t dbh = umma_desc(bhi + off, 128, (GKU / 4) * 128);
                    const uint64_t dbl = umma_desc(blo + off, 128, (GKU / 4) * 128);
                    umma_tf32_ss(dcol, dal, dbh, IDESC, q > 0);
                    umma_tf32_ss(dcol, dah, dbl, IDESC, 1);
                    umma_tf32_ss(dcol, dah, dbh, IDESC, 1);
                }
                umma_commit(&bdone[b]);
                umma_commit(&empty[sb]);
                // refill the buffer of the previous stage, whose MMAs were
                // issued one stage earlier
                if (s >= 1 && issued < nst) {
                    const int sp = s - 1;
                    if (!mbar_wait_abort(&empty[sp % GNST], (uint32_t)(sp / GNST) & 1u, abort, wait_ns)) break;
                    issue(issued++);
                }
            }
            umma_commit(&fin);
            mbar_wait_bounded(&fin, 0);
            for (int s = observed; s < issued; ++s)
                mbar_wait_bounded(&full[s % GNST], (uint32_t)(s / GNST) & 1u);
        }
        __syncwarp();
    } else {
        const int quarter = warp & 3, hf = warp >> 2;
        const uint32_t lane_off = (uint32_t)(quarter * 32) << 16;
        f2_t acc[FC / 2], cmp[FC / 2];
#pragma unroll
        for (int h = 0; h < FC / 2; ++h) acc[h] = cmp[h] = 0ull;
        auto fold = [&](int s) -> bool {
            if (!mbar_wait_abort_warp(&bdone[s & 1], (uint32_t)(s >> 1) & 1u, abort, wait_ns)) return false;
            tm_fence_after();
            const uint32_t dcol = tbase + lane_off + (s & 1) * NR + hf * FC;
            if constexpr (FC % 16 == 0) {
#pragma unroll
                for (int h = 0; h < FC / 16; ++h) {
                    uint32_t v[16];
                    tm_ld16(dcol + 16 * h, v);
                    umma_fold<16>(v, acc + 8 * h, cmp + 8 * h);
                }
            } else {
                uint32_t v[8];
                tm_ld8(dcol, v);
                umma_fold<8>(v, acc, cmp);
            }
            tm_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&dempty[s & 1]);
            return true;
        };
        bool ok = true;
        for (int s = 0; s < nst && ok; ++s) {
            const int sb = s % GNST;
            if (!mbar_wait_abort_warp(&full[sb], (uint32_t)(s / GNST) & 1u, abort, wait_ns)) {
                ok = false;
                break;
            }
            // split the raw tile in place into hi, and lo into the next buffer
            uint4 *raw = reinterpret_cast<uint4 *>(gsm + sb * SB);
            uint4 *lo = reinterpret_cast<uint4 *>(gsm + sb * SB + AB);
#pragma unroll 4
            for (int e = threadIdx.x; e < AB / 16; e += 256) {
                const uint4 v = raw[e];
                uint4 h, l;
                tf32_split(__uint_as_float(v.x), h.x, l.x);
                tf32_split(__uint_as_float(v.y), h.y, l.y);
                tf32_split(__uint_as_float(v.z), h.z, l.z);
                tf32_split(__uint_as_float(v.w), h.w, l.w);
                raw[e] = h;
                lo[e] = l;
            }
            // generic-proxy writes become visible to the tensor cores' reads
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(&split[sb]);
            if (s >= 1 && !fold(s - 1)) ok = false;
        }
        if (ok && nst > 0 && !fold(nst - 1)) ok = false;
        const int64_t i = rt * UR + quarter * 32 + lane;
        if (ok && i < M) {
#pragma unroll
            for (int h = 0; h < FC / 2; ++h) {
                float a0, a1;
                f2_unpack(acc[h], a0, a1);
                const int col = hf * FC + 2 * h;
                part[((int64_t)blockIdx.y * NR + col) * M + i] = a0;
                part[((int64_t)blockIdx.y * NR + col + 1) * M + i] = a1;
            }
        }
        tm_fence_before();
    }
    __syncthreads();
    if (warp == 8) {
        tm_fence_after();
        tm_dealloc(tbase, GU_TMEM);
    }
    if (threadIdx.x == 0 && *abort) atomicExch(err, DEV_TIMEOUT);
}

}  // namespace afn
