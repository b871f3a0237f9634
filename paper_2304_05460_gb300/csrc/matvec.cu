// matvec.cu -- matrix-free kernel matrix product q = (K + mu I) p
// (eq. (Problem): K_ij = K(x_i, x_j), never stored).
//
// Layout: each CTA owns TI = 64 rows i and one j-chunk of the points; its
// 256 threads are 4 j-groups x 64 rows.  Point tiles (TJ = 128 points) and
// the matching rows of p are staged in shared memory; every lane of a warp
// reads the same x_j (shared-memory broadcast).  A thread keeps its x_i and
// NR accumulators in registers; squared distance and the exponential are
// fused in registers.  The 4 j-groups are reduced in shared memory in a fixed
// order and each (row tile, j-chunk) CTA writes one partial; a second kernel
// sums the chunks in order and adds mu p.  The result is deterministic.
#include <algorithm>

#include "afn_device.cuh"
#include "afn_internal.cuh"

namespace afn {

static constexpr int TI = 64;       // rows per CTA
static constexpr int JG = 4;        // j-groups per CTA
static constexpr int TJ = 128;      // points per staged tile
static constexpr int NT = TI * JG;  // threads per CTA

int pad_dim(int d)
{
    if (d <= 3) return 3;
    if (d == 4) return 4;
    if (d <= 8) return 8;
    return 16;
}

static int num_sms()
{
    static int v = 0;
    if (!v) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
        if (v <= 0) v = 1;
    }
    return v;
}

// number of j-chunks: enough CTAs for several waves over all SMs, each chunk
// at least 4 tiles long.
static int pick_js(int64_t n)
{
    int64_t rt = (n + TI - 1) / TI;
    int64_t target = (int64_t)num_sms() * 6 * 4;
    int64_t js = (target + rt - 1) / rt;
    int64_t maxjs = std::max<int64_t>(1, (n + 4 * TJ - 1) / (4 * TJ));
    js = std::min<int64_t>(std::min<int64_t>(js, maxjs), 64);
    return (int)std::max<int64_t>(js, 1);
}

static void chunking(int64_t n, int &js, int64_t &chunk)
{
    js = pick_js(n);
    chunk = (n + js - 1) / js;
    chunk = (chunk + TJ - 1) / TJ * TJ;
    js = (int)((n + chunk - 1) / chunk);
}

static int piece(int left, int cap)
{
    int b = 1;
    while (b * 2 <= left && b * 2 <= cap) b *= 2;
    return b;
}

template <class T>
__global__ void matvec_finish(const T *__restrict__ part, int js, int nrc, int64_t n,
                              const T *__restrict__ P, int64_t ldp, T *__restrict__ Q,
                              int64_t ldq, T mu)
{
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n * nrc) return;
    int c = (int)(e / n);
    int64_t i = e % n;
    T s = 0;
    for (int q = 0; q < js; ++q) s += part[((int64_t)q * nrc + c) * n + i];
    Q[c * ldq + i] = s + mu * P[c * ldp + i];
}

// ------------------------------------------------------------------ FP32 --
// Xs: n x DS floats (DS = 4 when D == 3, else D), prescaled (kernel32_scaled).
template <int D, int NR, int KER>
__global__ void __launch_bounds__(NT) matvec32_kernel(const float *__restrict__ Xs, int64_t n,
                                                      const float *__restrict__ P, int64_t ldp,
                                                      float *__restrict__ part, int64_t chunk)
{
    constexpr int DS = (D == 3) ? 4 : D;
    constexpr int TILE = TJ * DS + NR * TJ;
    constexpr int RED = (JG - 1) * TI * NR;
    constexpr int SM = TILE > RED ? TILE : RED;
    __shared__ __align__(16) float sm[SM];
    float *xs = sm;
    float *ps = sm + TJ * DS;
    const int ti = threadIdx.x % TI;
    const int g = threadIdx.x / TI;
    const int64_t i = (int64_t)blockIdx.x * TI + ti;
    const int64_t j0 = (int64_t)blockIdx.y * chunk;
    const int64_t j1 = min(n, j0 + chunk);

    float xi[D];
#pragma unroll
    for (int t = 0; t < D; ++t) xi[t] = (i < n) ? Xs[i * DS + t] : 0.f;
    // two-level accumulation: a tile partial (TJ/JG terms) is folded into the
    // running sum with Kahan compensation, so the FP32 rounding of a row sum
    // grows like sqrt(TJ/JG) instead of sqrt(n / (JG * chunks)).
    float acc[NR], cmp[NR];
#pragma unroll
    for (int c = 0; c < NR; ++c) { acc[c] = 0.f; cmp[c] = 0.f; }

    for (int64_t jt = j0; jt < j1; jt += TJ) {
        __syncthreads();
        for (int e = threadIdx.x; e < TJ * DS; e += NT) {
            int64_t j = jt + e / DS;
            xs[e] = (j < j1) ? Xs[jt * DS + e] : 0.f;
        }
        for (int e = threadIdx.x; e < NR * TJ; e += NT) {
            int c = e / TJ, jj = e % TJ;
            int64_t j = jt + jj;
            ps[c * TJ + jj] = (j < j1) ? P[c * ldp + j] : 0.f;
        }
        __syncthreads();
        float tac[NR];
#pragma unroll
        for (int c = 0; c < NR; ++c) tac[c] = 0.f;
#pragma unroll 4
        for (int jj = g * (TJ / JG); jj < (g + 1) * (TJ / JG); ++jj) {
            const float *xj = xs + jj * DS;
            float r2 = 0.f;
#pragma unroll
            for (int t = 0; t < D; ++t) {
                float u = xi[t] - xj[t];
                r2 = fmaf(u, u, r2);
            }
            float kv = kernel32_scaled<KER>(r2);
#pragma unroll
            for (int c = 0; c < NR; ++c) tac[c] = fmaf(kv, ps[c * TJ + jj], tac[c]);
        }
#pragma unroll
        for (int c = 0; c < NR; ++c) {
            float y = tac[c] - cmp[c];
            float t = acc[c] + y;
            cmp[c] = (t - acc[c]) - y;
            acc[c] = t;
        }
    }
    __syncthreads();
    if (g > 0) {
#pragma unroll
        for (int c = 0; c < NR; ++c) sm[((g - 1) * NR + c) * TI + ti] = acc[c];
    }
    __syncthreads();
    if (g == 0 && i < n) {
#pragma unroll
        for (int c = 0; c < NR; ++c) {
            float s = acc[c];
            for (int q = 1; q < JG; ++q) s += sm[((q - 1) * NR + c) * TI + ti];
            part[((int64_t)blockIdx.y * NR + c) * n + i] = s;
        }
    }
}

// Packed variant for an even number of right-hand sides (NR in {2..32}):
// coordinates, distances and the NR accumulators are f32x2 pairs, x_j and
// p_j come from shared memory in 128-bit loads (p tile stored [j][c] with
// padded rows), so one j costs DS/4 + NR/4 shared loads and about
// DS + NR/2 + 4 FP32-pipe instructions.
template <int DS, int NR, int KER>
__global__ void __launch_bounds__(NT) matvec32p_kernel(const float *__restrict__ Xs, int64_t n,
                                                       const float *__restrict__ P, int64_t ldp,
                                                       float *__restrict__ part, int64_t chunk)
{
    constexpr int PS = (NR >= 4) ? NR + 4 : NR;          // p-tile row stride (floats)
    constexpr int TILE = TJ * DS + TJ * PS;
    constexpr int RED = (JG - 1) * TI * NR;
    constexpr int SM = TILE > RED ? TILE : RED;
    constexpr int H = NR / 2;
    __shared__ __align__(16) float sm[SM];
    float *xs = sm;
    float *ps = sm + TJ * DS;
    const int ti = threadIdx.x % TI;
    const int g = threadIdx.x / TI;
    const int64_t i = (int64_t)blockIdx.x * TI + ti;
    const int64_t j0 = (int64_t)blockIdx.y * chunk;
    const int64_t j1 = min(n, j0 + chunk);

    f2_t xi[DS / 2];
#pragma unroll
    for (int q = 0; q < DS / 2; ++q)
        xi[q] = (i < n) ? reinterpret_cast<const f2_t *>(Xs + i * DS)[q] : 0ull;
    // Kahan compensation of the tile folds costs NR more registers; above 16
    // right-hand sides it would halve occupancy, so it is kept only up to 16
    // (the two-level sum alone bounds the rounding growth by sqrt(TJ/JG) +
    // sqrt(tiles)).
    constexpr bool KAHAN = NR <= 16;
    f2_t acc[H], cmp[KAHAN ? H : 1];
#pragma unroll
    for (int c = 0; c < H; ++c) acc[c] = 0ull;
#pragma unroll
    for (int c = 0; c < (KAHAN ? H : 1); ++c) cmp[c] = 0ull;

    for (int64_t jt = j0; jt < j1; jt += TJ) {
        __syncthreads();
        for (int e = threadIdx.x; e < TJ * DS; e += NT) {
            int64_t j = jt + e / DS;
            xs[e] = (j < j1) ? Xs[jt * DS + e] : 0.f;
        }
        if (NR >= 4) {
            // each thread moves 4 consecutive columns of one j: coalesced global
            // reads per column, one conflict-free 128-bit shared store
            for (int e = threadIdx.x; e < TJ * NR / 4; e += NT) {
                int jj = e % TJ, c4 = e / TJ;
                int64_t j = jt + jj;
                float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
                if (j < j1) {
                    v.x = P[(4 * c4 + 0) * ldp + j];
                    v.y = P[(4 * c4 + 1) * ldp + j];
                    v.z = P[(4 * c4 + 2) * ldp + j];
                    v.w = P[(4 * c4 + 3) * ldp + j];
                }
                *reinterpret_cast<float4 *>(ps + jj * PS + 4 * c4) = v;
            }
        } else {
            for (int e = threadIdx.x; e < NR * TJ; e += NT) {
                int c = e / TJ, jj = e % TJ;
                int64_t j = jt + jj;
                ps[jj * PS + c] = (j < j1) ? P[c * ldp + j] : 0.f;
            }
        }
        __syncthreads();
        f2_t tac[H];
#pragma unroll
        for (int c = 0; c < H; ++c) tac[c] = 0ull;
#pragma unroll 2
        for (int jj = g * (TJ / JG); jj < (g + 1) * (TJ / JG); ++jj) {
            const ulonglong2 *xj = reinterpret_cast<const ulonglong2 *>(xs + jj * DS);
            f2_t r2p = 0ull;
#pragma unroll
            for (int q = 0; q < DS / 4; ++q) {
                ulonglong2 v = xj[q];
                f2_t u = f2_sub(xi[2 * q], v.x);
                r2p = f2_fma(u, u, r2p);
                u = f2_sub(xi[2 * q + 1], v.y);
                r2p = f2_fma(u, u, r2p);
            }
            float ra, rb;
            f2_unpack(r2p, ra, rb);
            const float kv = kernel32_scaled<KER>(ra + rb);
            const f2_t kv2 = f2_pack(kv, kv);
            if (NR >= 4) {
                const ulonglong2 *pj = reinterpret_cast<const ulonglong2 *>(ps + jj * PS);
#pragma unroll
                for (int q = 0; q < NR / 4; ++q) {
                    ulonglong2 pv = pj[q];
                    tac[2 * q] = f2_fma(kv2, pv.x, tac[2 * q]);
                    tac[2 * q + 1] = f2_fma(kv2, pv.y, tac[2 * q + 1]);
                }
            } else {
                tac[0] = f2_fma(kv2, *reinterpret_cast<const f2_t *>(ps + jj * PS), tac[0]);
            }
        }
        if constexpr (KAHAN) {
#pragma unroll
            for (int c = 0; c < H; ++c) {
                f2_t y = f2_sub(tac[c], cmp[c]);
                f2_t t = f2_add(acc[c], y);
                cmp[c] = f2_sub(f2_sub(t, acc[c]), y);
                acc[c] = t;
            }
        } else {
#pragma unroll
            for (int c = 0; c < H; ++c) acc[c] = f2_add(acc[c], tac[c]);
        }
    }
    __syncthreads();
    if (g > 0) {
#pragma unroll
        for (int c = 0; c < H; ++c) {
            float a, b;
            f2_unpack(acc[c], a, b);
            sm[((g - 1) * NR + 2 * c) * TI + ti] = a;
            sm[((g - 1) * NR + 2 * c + 1) * TI + ti] = b;
        }
    }
    __syncthreads();
    if (g == 0 && i < n) {
#pragma unroll
        for (int c = 0; c < H; ++c) {
            float a, b;
            f2_unpack(acc[c], a, b);
            for (int q = 1; q < JG; ++q) {
                a += sm[((q - 1) * NR + 2 * c) * TI + ti];
                b += sm[((q - 1) * NR + 2 * c + 1) * TI + ti];
            }
            part[((int64_t)blockIdx.y * NR + 2 * c) * n + i] = a;
            part[((int64_t)blockIdx.y * NR + 2 * c + 1) * n + i] = b;
        }
    }
}

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

template <int DS, int NB, int KER>
__global__ void __launch_bounds__(256, (2 * DS + 12 * NB + 24 <= 80) ? AFN_TC_MINB : 2)
    matvec32tc_kernel(const float *__restrict__ Xs, int64_t n, const float *__restrict__ P,
                      int64_t ldp, float *__restrict__ part, int64_t chunk)
{
    constexpr int NR = NB * 8;
    constexpr int PS = (NR == 8) ? 8 : (NR == 16 ? 24 : 40);   // t*PS distinct mod 32 by 8s
    constexpr int DSP = DS + 2;                                 // f2 stride of a point row
    __shared__ __align__(16) f2_t xsd[TCJ * DSP];               // (x, x) duplicated coordinates
    __shared__ __align__(16) uint32_t phi[TCJ * PS];
    __shared__ __align__(16) uint32_t plo[TCJ * PS];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = lane >> 2, t = lane & 3;
    const int64_t ia = (int64_t)blockIdx.x * TCR + warp * 16 + g;
    const int64_t ib = ia + 8;
    const int64_t j0 = (int64_t)blockIdx.y * chunk;
    const int64_t j1 = min(n, j0 + chunk);

    f2_t xi[DS];   // (x_ia[q], x_ib[q])
#pragma unroll
    for (int q = 0; q < DS; ++q)
        xi[q] = f2_pack(ia < n ? Xs[ia * DS + q] : 0.f, ib < n ? Xs[ib * DS + q] : 0.f);
    float acc[NB][4], cmp[TC_KAHAN ? NB : 1][4];
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
#pragma unroll
            for (int q = 0; q < DS; ++q) {
                f2_t u = f2_sub(xi[q], xa[q]);
                ra = f2_fma(u, u, ra);
                u = f2_sub(xi[q], xb[q]);
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
#pragma unroll
    for (int b = 0; b < NB; ++b) {
        const int c = b * 8 + 2 * t;
        float *p0 = part + ((int64_t)blockIdx.y * NR + c) * n;
        float *p1 = p0 + n;
        if (ia < n) { p0[ia] = acc[b][0]; p1[ia] = acc[b][1]; }
        if (ib < n) { p0[ib] = acc[b][2]; p1[ib] = acc[b][3]; }
    }
}

size_t matvec32_scratch(int64_t n, int nrhs)
{
    return sizeof(float) * (size_t)pick_js(n) * (size_t)std::min(std::max(nrhs, 1), 32) *
               (size_t)n + 256;
}

template <int D, int NR, int KER>
static void launch32(const float *Xs, int64_t n, const float *P, float *part, int js,
                     int64_t chunk, cudaStream_t s)
{
    dim3 grid((unsigned)((n + TI - 1) / TI), (unsigned)js);
#ifdef AFN_NO_TC
    constexpr bool use_tc = false;   // tuning build: CUDA-core kernels only
#else
    constexpr bool use_tc = true;
#endif
    if constexpr (NR >= 8 && use_tc) {
        dim3 gtc((unsigned)((n + TCR - 1) / TCR), (unsigned)js);
        matvec32tc_kernel<(D == 3 ? 4 : D), NR / 8, KER><<<gtc, 256, 0, s>>>(Xs, n, P, n, part, chunk);
    } else if constexpr (NR >= 2) {
        matvec32p_kernel<(D == 3 ? 4 : D), NR, KER><<<grid, NT, 0, s>>>(Xs, n, P, n, part, chunk);
    } else {
        matvec32_kernel<D, NR, KER><<<grid, NT, 0, s>>>(Xs, n, P, n, part, chunk);
    }
}

template <int D, int KER>
static void launch32_nr(int nr, const float *Xs, int64_t n, const float *P, float *part, int js,
                        int64_t chunk, cudaStream_t s)
{
    switch (nr) {
    case 1: launch32<D, 1, KER>(Xs, n, P, part, js, chunk, s); break;
    case 2: launch32<D, 2, KER>(Xs, n, P, part, js, chunk, s); break;
    case 4: launch32<D, 4, KER>(Xs, n, P, part, js, chunk, s); break;
    case 8: launch32<D, 8, KER>(Xs, n, P, part, js, chunk, s); break;
    case 16: launch32<D, 16, KER>(Xs, n, P, part, js, chunk, s); break;
    default: launch32<D, 32, KER>(Xs, n, P, part, js, chunk, s); break;
    }
}

template <int KER>
static void launch32_d(int dp, int nr, const float *Xs, int64_t n, const float *P, float *part,
                       int js, int64_t chunk, cudaStream_t s)
{
    switch (dp) {
    case 3: launch32_nr<3, KER>(nr, Xs, n, P, part, js, chunk, s); break;
    case 4: launch32_nr<4, KER>(nr, Xs, n, P, part, js, chunk, s); break;
    case 8: launch32_nr<8, KER>(nr, Xs, n, P, part, js, chunk, s); break;
    default: launch32_nr<16, KER>(nr, Xs, n, P, part, js, chunk, s); break;
    }
}

// p, q: n x nrhs column-major with leading dimension n.
afn_status matvec32(const float *Xs, int64_t n, int dp, int kernel, float mu, const float *p,
                    int nrhs, float *q, void *scratch, size_t scratch_bytes, cudaStream_t s)
{
    if (n <= 0 || nrhs <= 0) return AFN_OK;
    if (scratch_bytes < matvec32_scratch(n, nrhs)) {
        set_error("matvec32: scratch too small");
        return AFN_ERR_ARG;
    }
    int js;
    int64_t chunk;
    chunking(n, js, chunk);
    float *part = static_cast<float *>(scratch);
    for (int c0 = 0; c0 < nrhs;) {
#ifdef AFN_NO_TC
        int b = piece(nrhs - c0, 16);
#else
        int b = piece(nrhs - c0, 32);
#endif
        const float *pp = p + (int64_t)c0 * n;
        if (kernel == 0) launch32_d<0>(dp, b, Xs, n, pp, part, js, chunk, s);
        else launch32_d<1>(dp, b, Xs, n, pp, part, js, chunk, s);
        int64_t tot = n * b;
        matvec_finish<float><<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(
            part, js, b, n, pp, n, q + (int64_t)c0 * n, n, mu);
        c0 += b;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "matvec32 launch");
    return AFN_OK;
}

// ------------------------------------------------------------------ FP64 --
template <int D, int NR>
__global__ void __launch_bounds__(NT) matvec64_kernel(const double *__restrict__ X, int d,
                                                      int64_t n, int kernel, double l,
                                                      const double *__restrict__ P, int64_t ldp,
                                                      double *__restrict__ part, int64_t chunk)
{
    constexpr int TILE = TJ * D + NR * TJ;
    constexpr int RED = (JG - 1) * TI * NR;
    constexpr int SM = TILE > RED ? TILE : RED;
    __shared__ double sm[SM];
    double *xs = sm;
    double *ps = sm + TJ * D;
    const int ti = threadIdx.x % TI;
    const int g = threadIdx.x / TI;
    const int64_t i = (int64_t)blockIdx.x * TI + ti;
    const int64_t j0 = (int64_t)blockIdx.y * chunk;
    const int64_t j1 = min(n, j0 + chunk);
    double xi[D];
#pragma unroll
    for (int t = 0; t < D; ++t) xi[t] = (i < n && t < d) ? X[i * d + t] : 0.0;
    double acc[NR];
#pragma unroll
    for (int c = 0; c < NR; ++c) acc[c] = 0.0;
    const double inv_l2 = 1.0 / (l * l);
    const double s3l = 1.7320508075688772 / l;
    for (int64_t jt = j0; jt < j1; jt += TJ) {
        __syncthreads();
        for (int e = threadIdx.x; e < TJ * D; e += NT) {
            int jj = e / D, t = e % D;
            int64_t j = jt + jj;
            xs[e] = (j < j1 && t < d) ? X[j * d + t] : 0.0;
        }
        for (int e = threadIdx.x; e < NR * TJ; e += NT) {
            int c = e / TJ, jj = e % TJ;
            int64_t j = jt + jj;
            ps[c * TJ + jj] = (j < j1) ? P[c * ldp + j] : 0.0;
        }
        __syncthreads();
        for (int jj = g * (TJ / JG); jj < (g + 1) * (TJ / JG); ++jj) {
            const double *xj = xs + jj * D;
            double r2 = 0.0;
#pragma unroll
            for (int t = 0; t < D; ++t) {
                double u = xi[t] - xj[t];
                r2 = fma(u, u, r2);
            }
            double kv;
            if (kernel == 0) {
                kv = exp(-r2 * inv_l2);
            } else {
                double tt = sqrt(r2) * s3l;
                kv = (1.0 + tt) * exp(-tt);
            }
#pragma unroll
            for (int c = 0; c < NR; ++c) acc[c] = fma(kv, ps[c * TJ + jj], acc[c]);
        }
    }
    __syncthreads();
    if (g > 0) {
#pragma unroll
        for (int c = 0; c < NR; ++c) sm[((g - 1) * NR + c) * TI + ti] = acc[c];
    }
    __syncthreads();
    if (g == 0 && i < n) {
#pragma unroll
        for (int c = 0; c < NR; ++c) {
            double s = acc[c];
            for (int q = 1; q < JG; ++q) s += sm[((q - 1) * NR + c) * TI + ti];
            part[((int64_t)blockIdx.y * NR + c) * n + i] = s;
        }
    }
}

size_t matvec64_scratch(int64_t n, int nrhs)
{
    return sizeof(double) * (size_t)pick_js(n) * (size_t)std::min(std::max(nrhs, 1), 32) *
               (size_t)n + 256;
}

template <int D>
static void launch64_nr(int nr, const double *X, int d, int64_t n, int kernel, double l,
                        const double *P, double *part, int js, int64_t chunk, cudaStream_t s)
{
    dim3 grid((unsigned)((n + TI - 1) / TI), (unsigned)js);
    switch (nr) {
    case 1: matvec64_kernel<D, 1><<<grid, NT, 0, s>>>(X, d, n, kernel, l, P, n, part, chunk); break;
    case 2: matvec64_kernel<D, 2><<<grid, NT, 0, s>>>(X, d, n, kernel, l, P, n, part, chunk); break;
    case 4: matvec64_kernel<D, 4><<<grid, NT, 0, s>>>(X, d, n, kernel, l, P, n, part, chunk); break;
    case 8: matvec64_kernel<D, 8><<<grid, NT, 0, s>>>(X, d, n, kernel, l, P, n, part, chunk); break;
    case 16: matvec64_kernel<D, 16><<<grid, NT, 0, s>>>(X, d, n, kernel, l, P, n, part, chunk); break;
    default: matvec64_kernel<D, 32><<<grid, NT, 0, s>>>(X, d, n, kernel, l, P, n, part, chunk); break;
    }
}

afn_status matvec64(const double *X, int64_t n, int d, KParams kp, const double *p, int nrhs,
                    double *q, void *scratch, size_t scratch_bytes, cudaStream_t s)
{
    if (n <= 0 || nrhs <= 0) return AFN_OK;
    if (scratch_bytes < matvec64_scratch(n, nrhs)) {
        set_error("matvec64: scratch too small");
        return AFN_ERR_ARG;
    }
    int js;
    int64_t chunk;
    chunking(n, js, chunk);
    double *part = static_cast<double *>(scratch);
    int dpad = pad_dim(d);
    for (int c0 = 0; c0 < nrhs;) {
        int b = piece(nrhs - c0, 32);
        const double *pp = p + (int64_t)c0 * n;
        switch (dpad) {
        case 3: launch64_nr<3>(b, X, d, n, kp.kernel, kp.l, pp, part, js, chunk, s); break;
        case 4: launch64_nr<4>(b, X, d, n, kp.kernel, kp.l, pp, part, js, chunk, s); break;
        case 8: launch64_nr<8>(b, X, d, n, kp.kernel, kp.l, pp, part, js, chunk, s); break;
        default: launch64_nr<16>(b, X, d, n, kp.kernel, kp.l, pp, part, js, chunk, s); break;
        }
        int64_t tot = n * b;
        matvec_finish<double><<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(
            part, js, b, n, pp, n, q + (int64_t)c0 * n, n, kp.mu);
        c0 += b;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "matvec64 launch");
    return AFN_OK;
}

// --------------------------------------------------- FP32 point staging --
// Prescaled coordinates x~ = fl32(x * scale), n x ds (ds = stored_dim32(dp)).
__global__ void points32_kernel(const double *__restrict__ X, int64_t n, int d, int ds,
                                double scale, float *__restrict__ Xs)
{
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n * ds) return;
    int64_t i = e / ds;
    int t = (int)(e % ds);
    Xs[e] = (t < d) ? (float)(X[i * d + t] * scale) : 0.f;
}

int stored_dim32(int dp) { return dp == 3 ? 4 : dp; }

afn_status make_points32(const double *X, int64_t n, int d, int dp, int kernel, double l,
                         float *Xs, cudaStream_t s)
{
    int ds = stored_dim32(dp);
    double scale = (kernel == 0) ? 1.2011224087864498 / l   // sqrt(log2 e) / l
                                 : 1.7320508075688772 / l;  // sqrt(3) / l
    int64_t tot = n * ds;
    if (tot == 0) return AFN_OK;
    points32_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(X, n, d, ds, scale, Xs);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "points32 launch");
    return AFN_OK;
}

}  // namespace afn
