// gemm_bf16.cuh -- the two W products of the FP32 preconditioner apply
// (Alg. 3) on the fifth-generation tensor cores with BF16 operands:
//   t = r2 - W^T z'   (rows i of W^T, K = the k landmarks)
//   u = z' - W s2     (rows p of W,   K = the n_r remaining points)
// The operand matrix is rounded to BF16 once per build and stored in a tiled
// image (row tile of 128 x stage of GKB K-elements, the K-major core-matrix
// layout of the MMA), half the bytes of the FP32 copy, so each stage is one
// contiguous bulk copy and the products stream half the HBM traffic.  The
// vector block keeps (nearly) FP32 accuracy: each value is split into NT
// BF16 terms, v = t_0 + t_1 (+ t_2), and the terms sit side by side along N,
// so one MMA per K-step forms A [B_0 | B_1 | B_2] and the epilogue adds the
// term columns.  Accumulation is FP32 in tensor memory over the CTA's whole
// K-chunk; chunk partials are summed in a fixed order by gemm_finish.
//
// CTA = 5 warps: warps 0-3 own TMEM lane quarters and run the epilogue, warp
// 4 owns the TMEM allocation and one of its threads issues the bulk copies
// and the MMAs.  Stages rotate through GBNST buffers; an MMA commit frees a
// buffer for the next copy.  Every wait is bounded (the wait limit, 2 s by
// default) with a CTA-wide abort flag; the drain after an abort waits up to
// 2 s for copies and MMAs in flight.
//
// Layouts (bytes; a core matrix is 8 rows x 16 bytes = 8 x 8 BF16):
//   A stage: core matrix (r / 8, kk / 8) at ((r / 8) (GKB / 8) + kk / 8) 128,
//            row r % 8 at 16 (r % 8), element kk % 8 at 2 (kk % 8);
//   B stage: the same with the column n' = term NC + c in place of r.
// MMA descriptors: leading byte offset 128 (next core matrix along K),
// stride byte offset (GKB / 8) 128 (next 8 rows / columns); a K-step of 16
// elements advances the start address by 256 bytes.
#pragma once

#include <cuda_bf16.h>

#include "matvec_umma.cuh"

namespace afn {

static constexpr int GKB = 64;      // K-elements per stage (4 MMA k-steps of 16)
static constexpr int GBNST = 4;     // stage buffers
static constexpr int GBT = 160;     // threads: 4 epilogue warps + 1 issuing warp
static constexpr int GB_TMEM = 256; // accumulator columns allocated (>= NT NC)

template <int NC, int NT> struct GbStage {
    static constexpr int NP = NC * NT;                 // MMA N (term columns)
    static constexpr int AB = UR * GKB * 2;            // A tile bytes (16 KB)
    static constexpr int BB = GKB * NP * 2;            // B tile bytes
    static constexpr int BYTES = AB + BB;
};

// element index of (row r, K-element kk) inside one 128 x GKB stage tile
__host__ __device__ inline int64_t gb_tile_elem(int r, int kk)
{
    return (int64_t)((r / 8) * (GKB / 8) + kk / 8) * 64 + (r % 8) * 8 + (kk % 8);
}

// instruction descriptor: D f32, A and B bf16 (both K-major), M x N
__host__ __device__ constexpr uint32_t umma_idesc_bf16(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}

// D (+)= A B, kind::f16 (bf16 operands), both operands described in shared memory
__device__ __forceinline__ void umma_bf16_ss(uint32_t dt, uint64_t adesc, uint64_t bdesc,
                                             uint32_t idesc, uint32_t accumulate)
{
    asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                 " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(dt),
                 "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
                 : "memory");
}

// part[(y NC + c) M + i] = sum over the CTA's stages of A[i, :] v[:, c] for
// the 128 rows of row tile blockIdx.x.  Atl: the BF16 image (row tiles of
// nks stages, UR * GKB elements a stage); Bk: the split vector block (per
// stage GKB x NT NC BF16 in the layout above).
template <int NC, int NT>
__global__ void __launch_bounds__(GBT, 1)
    gemm16u_kernel(const __nv_bfloat16 *__restrict__ Atl, int64_t M, int64_t nks,
                   const __nv_bfloat16 *__restrict__ Bk, float *__restrict__ part,
                   int64_t chunk_st, int *__restrict__ err, uint64_t wait_ns)
{
    constexpr int NP = GbStage<NC, NT>::NP;
    constexpr int AB = GbStage<NC, NT>::AB, BB = GbStage<NC, NT>::BB;
    constexpr int SB = GbStage<NC, NT>::BYTES;
    constexpr uint32_t IDESC = umma_idesc_bf16(UR, NP);
    static_assert(NP % 16 == 0 && NP <= GB_TMEM && NC % 16 == 0, "shape");

    extern __shared__ __align__(128) unsigned char gbsm[];
    __shared__ __align__(8) uint64_t full[GBNST], empty[GBNST], fin;
    __shared__ uint32_t tbase_slot;
    __shared__ int abort_flag;
    volatile int *abort = &abort_flag;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t rt = blockIdx.x;
    const int64_t s0 = (int64_t)blockIdx.y * chunk_st;
    const int nst = (int)(min(nks, s0 + chunk_st) - s0);

    if (threadIdx.x == 0) {
        for (int b = 0; b < GBNST; ++b) {
            mbar_init(&full[b], 1);
            mbar_init(&empty[b], 1);
        }
        mbar_init(&fin, 1);
        abort_flag = 0;
        mbar_init_fence();
    }
    if (warp == 4) tm_alloc(&tbase_slot, GB_TMEM);
    tm_fence_before();
    __syncthreads();
    tm_fence_after();
    const uint32_t tbase = tbase_slot;

    if (warp == 4) {
        if (lane == 0) {
            int issued = 0, observed = 0;
            auto issue = [&](int s) {
                unsigned char *st = gbsm + (s % GBNST) * SB;
                uint64_t *bar = &full[s % GBNST];
                mbar_expect_tx(bar, (uint32_t)SB);
                bulk_g2s(st, Atl + (rt * nks + s0 + s) * (int64_t)(UR * GKB), (uint32_t)AB, bar);
                bulk_g2s(st + AB, Bk + (s0 + s) * (int64_t)(GKB * NP), (uint32_t)BB, bar);
            };
            for (; issued < nst && issued < GBNST; ++issued) issue(issued);
            const uint32_t base_s = smem_addr(gbsm);
            for (int s = 0; s < nst && !*abort; ++s) {
                const int sb = s % GBNST;
                if (!mbar_wait_abort(&full[sb], (uint32_t)(s / GBNST) & 1u, abort, wait_ns)) break;
                observed = s + 1;
                tm_fence_after();
                const uint32_t a0 = base_s + sb * SB, b0 = a0 + AB;
#pragma unroll
                for (int q = 0; q < GKB / 16; ++q) {
                    const uint64_t da = umma_desc(a0 + q * 256, 128, (GKB / 8) * 128);
                    const uint64_t db = umma_desc(b0 + q * 256, 128, (GKB / 8) * 128);
                    umma_bf16_ss(tbase, da, db, IDESC, (s > 0 || q > 0) ? 1u : 0u);
                }
                umma_commit(&empty[sb]);
                // refill the buffer of the previous stage, whose MMAs were
                // issued one stage earlier
                if (s >= 1 && issued < nst) {
                    const int sp = s - 1;
                    if (!mbar_wait_abort(&empty[sp % GBNST], (uint32_t)(sp / GBNST) & 1u, abort, wait_ns))
                        break;
                    issue(issued++);
                }
            }
            umma_commit(&fin);
            // drain (bounded): every MMA issued so far, then every copy whose
            // completion this thread has not observed
            mbar_wait_bounded(&fin, 0);
            for (int s = observed; s < issued; ++s)
                mbar_wait_bounded(&full[s % GBNST], (uint32_t)(s / GBNST) & 1u);
        }
        __syncwarp();
    } else {
        // epilogue: row i of the tile is TMEM lane i; columns t NC + c
        const bool ok = nst > 0 && mbar_wait_abort_warp(&fin, 0u, abort, wait_ns) && !*abort;
        tm_fence_after();
        const int64_t i = rt * UR + warp * 32 + lane;
        const uint32_t lane_off = (uint32_t)(warp * 32) << 16;
        if (nst == 0 && i < M) {
            for (int c = 0; c < NC; ++c) part[((int64_t)blockIdx.y * NC + c) * M + i] = 0.f;
        }
        if (__all_sync(0xffffffffu, ok)) {
#pragma unroll
            for (int c16 = 0; c16 < NC / 16; ++c16) {
                float acc[16];
                uint32_t v[16];
                tm_ld16(tbase + lane_off + (NT - 1) * NC + 16 * c16, v);
#pragma unroll
                for (int e = 0; e < 16; ++e) acc[e] = __uint_as_float(v[e]);
#pragma unroll
                for (int t = NT - 2; t >= 0; --t) {
                    tm_ld16(tbase + lane_off + t * NC + 16 * c16, v);
#pragma unroll
                    for (int e = 0; e < 16; ++e) acc[e] += __uint_as_float(v[e]);
                }
                if (i < M) {
#pragma unroll
                    for (int e = 0; e < 16; ++e)
                        part[((int64_t)blockIdx.y * NC + 16 * c16 + e) * M + i] = acc[e];
                }
            }
        }
        tm_fence_before();
    }
    __syncthreads();
    if (warp == 4) {
        tm_fence_after();
        tm_dealloc(tbase, GB_TMEM);
    }
    if (threadIdx.x == 0 && *abort) atomicExch(err, DEV_TIMEOUT);
}

}  // namespace afn
