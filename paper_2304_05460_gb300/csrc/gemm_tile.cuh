// gemm_tile.cuh -- the register-tiled product tile used by the AFN apply
// (apply.cu) for one system and by the grouped apply of many systems.
#pragma once

#include <stdint.h>

namespace afn {

static constexpr int GM = 128;     // output rows per CTA
static constexpr int GK = 16;      // K per shared-memory stage

template <int NC> struct GemmShape {
    static constexpr int TC = NC / 4;          // threads along columns
    static constexpr int TR = 256 / TC;        // threads along rows
    static constexpr int RM = GM / TR;         // rows per thread
};

// acc = op(A)[r0:r0+GM, k0:k1] X[k0:k1, 0:NC] for a 256-thread CTA:
//   TA == false: op(A) = A, A row-major M x K   (A[i,p] = A[i*lda+p])
//   TA == true : op(A) = A^T, A row-major K x M (A^T[i,p] = A[p*lda+i])
// X column-major with leading dimension ldx.  TRI = 1 keeps only p <= i
// (lower), TRI = 2 only p >= i (upper).  Thread (tr, tc) = (threadIdx.x /
// TC, threadIdx.x % TC) owns rows r0 + tr*RM + a and columns tc*4 + b.
template <class T, int NC, bool TA, int TRI>
__device__ __forceinline__ void gemm_rows(const T *__restrict__ A, int64_t lda, int64_t M,
                                          int64_t r0, int64_t k0, int64_t k1,
                                          const T *__restrict__ X, int64_t ldx,
                                          T (&as)[GK][GM + 4], T (&xs)[GK][NC + 4],
                                          T (&acc)[GemmShape<NC>::RM][4])
{
    constexpr int TC = NC / 4;             // threads along columns
    constexpr int TR = 256 / TC;           // threads along rows
    constexpr int RM = GM / TR;            // rows per thread
    const int tc = threadIdx.x % TC, tr = threadIdx.x / TC;
    if (TRI == 1) k1 = min(k1, r0 + GM);          // p <= i <= r0 + GM - 1
    if (TRI == 2) k0 = max(k0, r0);               // p >= i >= r0
#pragma unroll
    for (int a = 0; a < RM; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = 0;
    // register prefetch: the next stage's global loads are issued before the
    // current stage is computed
    constexpr int LA = GM * GK / 256;                        // A elements per thread
    constexpr int LX = (GK * NC + 255) / 256;                // X elements per thread
    T ra[LA], rx[LX];
    auto fetch = [&](int64_t kk0) {
#pragma unroll
        for (int u = 0; u < LA; ++u) {
            int e = threadIdx.x + u * 256;
            int r, q;
            if (TA) { q = e / GM; r = e % GM; }       // coalesced along i
            else { r = e / GK; q = e % GK; }          // coalesced along p
            int64_t gi = r0 + r, gp = kk0 + q;
            T v = 0;
            if (gi < M && gp < k1) {
                bool keep = (TRI == 0) || (TRI == 1 && gp <= gi) || (TRI == 2 && gp >= gi);
                if (keep) v = TA ? A[gp * lda + gi] : A[gi * lda + gp];
            }
            ra[u] = v;
        }
#pragma unroll
        for (int u = 0; u < LX; ++u) {
            int e = threadIdx.x + u * 256;
            int c = e / GK, q = e % GK;
            int64_t gp = kk0 + q;
            rx[u] = (e < GK * NC && gp < k1) ? X[c * ldx + gp] : (T)0;
        }
    };
    if (k0 < k1) fetch(k0);
    for (int64_t kk0 = k0; kk0 < k1; kk0 += GK) {
        __syncthreads();
#pragma unroll
        for (int u = 0; u < LA; ++u) {
            int e = threadIdx.x + u * 256;
            int r, q;
            if (TA) { q = e / GM; r = e % GM; }
            else { r = e / GK; q = e % GK; }
            as[q][r] = ra[u];
        }
#pragma unroll
        for (int u = 0; u < LX; ++u) {
            int e = threadIdx.x + u * 256;
            if (e < GK * NC) xs[e % GK][e / GK] = rx[u];
        }
        __syncthreads();
        if (kk0 + GK < k1) fetch(kk0 + GK);
#pragma unroll
        for (int q = 0; q < GK; ++q) {
            T av[RM], xv[4];
#pragma unroll
            for (int a = 0; a < RM; ++a) av[a] = as[q][tr * RM + a];
#pragma unroll
            for (int b = 0; b < 4; ++b) xv[b] = xs[q][tc * 4 + b];
#pragma unroll
            for (int a = 0; a < RM; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) acc[a][b] += av[a] * xv[b];
        }
    }
}

}  // namespace afn
