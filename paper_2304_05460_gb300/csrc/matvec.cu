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
#include <atomic>
#include <cstring>
#include <type_traits>

#include "afn_device.cuh"
#include "afn_internal.cuh"
#include "matvec_tc.cuh"
#include "matvec_umma.cuh"
#include "matvec_df.cuh"
#include "group.cuh"

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

// One right-hand side, two rows per thread: the rows i and i + 64 of a
// 128-row CTA share every staged x_j and p_j, and their distances, kernel
// arguments and sums are f32x2 pairs (each half rounded as the scalar
// operation).  The staged tile holds each coordinate and p_j twice,
// {v, v}, so a packed operand is one shared load.  Per row: r^2 by FMAs over
// d ascending, the j-group's partial over j ascending, folded into the running
// sum with Kahan compensation once per staged tile (so the FP32 rounding of a
// row sum grows like sqrt(TJ/JG), not sqrt(n/JG)), j-groups summed in order.
static constexpr int TI2 = 2 * TI;   // rows per CTA of the two-row form

template <int D, int KER>
__global__ void __launch_bounds__(NT) matvec32r2_kernel(const float *__restrict__ Xs, int64_t n,
                                                        const float *__restrict__ P,
                                                        float *__restrict__ part, int64_t chunk)
{
    constexpr int DS = (D == 3) ? 4 : D;
    constexpr int TILE = TJ * D + TJ;                 // f2_t entries: coordinates, then p
    __shared__ __align__(16) f2_t sm2[TILE];
    f2_t *xs = sm2;
    f2_t *ps = sm2 + TJ * D;
    const int ti = threadIdx.x % TI;
    const int g = threadIdx.x / TI;
    const int64_t i0 = (int64_t)blockIdx.x * TI2 + ti, i1 = i0 + TI;
    const int64_t j0 = (int64_t)blockIdx.y * chunk;
    const int64_t j1 = min(n, j0 + chunk);

    f2_t xi[D];
#pragma unroll
    for (int t = 0; t < D; ++t)
        xi[t] = f2_pack(i0 < n ? Xs[i0 * DS + t] : 0.f, i1 < n ? Xs[i1 * DS + t] : 0.f);
    f2_t acc = 0ull, cmp = 0ull;
    for (int64_t jt = j0; jt < j1; jt += TJ) {
        __syncthreads();
        for (int e = threadIdx.x; e < TJ * D; e += NT) {
            const int jj = e / D, t = e % D;
            const int64_t j = jt + jj;
            const float v = j < j1 ? Xs[j * DS + t] : 0.f;
            xs[e] = f2_pack(v, v);
        }
        for (int jj = threadIdx.x; jj < TJ; jj += NT) {
            const int64_t j = jt + jj;
            const float v = j < j1 ? P[j] : 0.f;
            ps[jj] = f2_pack(v, v);
        }
        __syncthreads();
        f2_t tac = 0ull;
#pragma unroll 4
        for (int jj = g * (TJ / JG); jj < (g + 1) * (TJ / JG); ++jj) {
            const f2_t *xj = xs + jj * D;
            f2_t r2 = 0ull;
#pragma unroll
            for (int t = 0; t < D; ++t) {
                const f2_t u = f2_sub(xi[t], xj[t]);
                r2 = f2_fma(u, u, r2);
            }
            float ra, rb;
            f2_unpack(r2, ra, rb);
            tac = f2_fma(f2_pack(kernel32_scaled<KER>(ra), kernel32_scaled<KER>(rb)), ps[jj], tac);
        }
        const f2_t y = f2_sub(tac, cmp);
        const f2_t t2 = f2_add(acc, y);
        cmp = f2_sub(f2_sub(t2, acc), y);
        acc = t2;
    }
    __syncthreads();
    float *red = reinterpret_cast<float *>(sm2);
    float a0, a1;
    f2_unpack(acc, a0, a1);
    if (g > 0) {
        red[((g - 1) * 2 + 0) * TI + ti] = a0;
        red[((g - 1) * 2 + 1) * TI + ti] = a1;
    }
    __syncthreads();
    if (g == 0) {
        float s0 = a0, s1 = a1;
        for (int q = 1; q < JG; ++q) {
            s0 += red[((q - 1) * 2 + 0) * TI + ti];
            s1 += red[((q - 1) * 2 + 1) * TI + ti];
        }
        if (i0 < n) part[(int64_t)blockIdx.y * n + i0] = s0;
        if (i1 < n) part[(int64_t)blockIdx.y * n + i1] = s1;
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

// Single-system mma.sync tensor-core kernel: CTA = 128 rows x one j-chunk with
// TMA-staged, double-buffered tiles (mv32tc_rows_async) read from the prepared
// Xdup / Psp arrays; one partial per (chunk, column), summed in order by
// matvec_finish.
template <int DS, int NB, int KER>
__global__ void __launch_bounds__(256, (2 * DS + 12 * NB + 24 <= 80) ? TC_MINB : 2)
    matvec32tca_kernel(const float *__restrict__ Xs, int64_t n, const f2_t *__restrict__ Xdup,
                       const uint32_t *__restrict__ Psp, float *__restrict__ part, int64_t chunk,
                       int *__restrict__ err)
{
    constexpr int NR = NB * 8;
    extern __shared__ __align__(16) unsigned char dsm[];
    __shared__ __align__(8) uint64_t bars[2];
    if (threadIdx.x == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        mbar_init_fence();
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = lane >> 2, t = lane & 3;
    const int64_t ia = (int64_t)blockIdx.x * TCR + warp * 16 + g;
    const int64_t ib = ia + 8;
    const int64_t j0 = (int64_t)blockIdx.y * chunk;
    const int64_t j1 = min(n, j0 + chunk);
    float acc[NB][4];
    uint32_t parity = 0;
    if (!mv32tc_rows_async<DS, NB, KER>(Xs, n, Xdup, Psp, (int64_t)blockIdx.x * TCR, j0, j1, dsm,
                                        bars, parity, acc)) {
        if (threadIdx.x == 0) atomicExch(err, DEV_TIMEOUT);
        return;
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

// Xdup: rows of (x, x) pairs, DS + 2 per row, zero rows up to npad
__global__ void dup_points_kernel(const float *__restrict__ Xs, int64_t n, int ds, int64_t npad,
                                  f2_t *__restrict__ Xdup)
{
    const int dsp = ds + 2;
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= npad * dsp) return;
    const int64_t j = e / dsp;
    const int q = (int)(e % dsp);
    const float v = (j < n && q < ds) ? Xs[j * ds + q] : 0.f;
    Xdup[e] = f2_pack(v, v);
}

// Psp: row j = [tf32 hi of p(j, c), c < NR | pad | lo | pad], zero rows up to npad
template <int NB>
__global__ void psplit_kernel(const float *__restrict__ P, int64_t ldp, int64_t n, int64_t npad,
                              uint32_t *__restrict__ Psp)
{
    constexpr int NR = NB * 8;
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= npad * NR) return;
    const int64_t j = e % npad;
    const int c = (int)(e / npad);
    uint32_t hi, lo;
    tf32_split(j < n ? P[c * ldp + j] : 0.f, hi, lo);
    Psp[j * TcRow<NB>::ROW + c] = hi;
    Psp[j * TcRow<NB>::ROW + TcRow<NB>::PS + c] = lo;
}

static int64_t tc_npad(int64_t n) { return (n + TCJ - 1) / TCJ * TCJ; }
static_assert(TCJ % UJ == 0, "the prepared arrays of both tensor-core paths share npad");

// Xpr: per stage of UJ points, the point tile of matvec32u_kernel for the
// distance form VAR (zero rows up to npad); the norms are the FMA chain the
// kernel uses for its dot products
// Xpr: per stage of UJ points, the pairs (2m + h, q) at float 2m ds + 2q + h
// (two points per f32x2 operand), zero rows up to npad
__global__ void upoints_kernel(const float *__restrict__ Xs, int64_t n, int ds, int64_t npad,
                               float *__restrict__ Xpr)
{
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= npad) return;
    const int64_t base = (j / UJ) * (int64_t)UJ * ds;
    const int jj = (int)(j % UJ);
    for (int q = 0; q < ds; ++q) {
        const float v = j < n ? Xs[j * ds + q] : 0.f;
        Xpr[base + (int64_t)(jj & ~1) * ds + 2 * q + (jj & 1)] = v;
    }
}

// Pk: per stage of UJ points, the tf32 hi then lo halves of p in the K-major
// core-matrix layout of matvec32u_kernel, zero rows up to npad
template <int NR>
__global__ void ksplit_kernel(const float *__restrict__ P, int64_t ldp, int64_t n, int64_t npad,
                              uint32_t *__restrict__ Pk)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= npad * NR) return;
    const int64_t j = e % npad;
    const int c = (int)(e / npad);
    uint32_t hi, lo;
    tf32_split(j < n ? P[c * ldp + j] : 0.f, hi, lo);
    const int64_t st = j / UJ;
    const int jj = (int)(j % UJ);
    const int64_t w = st * (2 * UJ * NR) + (c / 8) * (UJ / 4) * 32 + (jj / 4) * 32 + (c % 8) * 4 +
                      (jj % 4);
    Pk[w] = hi;
    Pk[w + UJ * NR] = lo;
}

static constexpr int UJS_MAX = 8;   // j-chunks of the tcgen05 path

// j-chunks (in staged tiles) of the tcgen05 path: the count whose CTAs fill
// the last wave of 2 CTAs per SM best, chunks of at least 4 tiles
static void chunking_u(int64_t n, int64_t nstage, int &js, int64_t &chunk_st)
{
    const int64_t rt = (n + UR - 1) / UR;
    const int64_t slots = 2 * (int64_t)num_sms();
    double best = -1.0;
    js = 1;
    chunk_st = nstage;
    for (int q = 1; q <= UJS_MAX; ++q) {
        const int64_t cs = (nstage + q - 1) / q;
        if (q > 1 && cs < 4) break;
        const int64_t jq = (nstage + cs - 1) / cs;
        const int64_t tot = rt * jq;
        const int64_t waves = (tot + slots - 1) / slots;
        const double eff = (double)tot / (double)(waves * slots);
        if (eff > best + 1e-9) {
            best = eff;
            js = (int)jq;
            chunk_st = cs;
        }
    }
}

template <int DS, int NB, int KER, int UH>
static void launch_u(const float *Xs, int64_t n, const float *Xpr, const uint32_t *Pk, float *part,
                     int js, int64_t chunk_st, int64_t nstage, int *err, cudaStream_t s)
{
    // at least 80 KB of shared memory keeps residency at 2 CTAs per SM, the
    // number whose tensor-memory allocations fit together
    const int smem = std::max(UNST * UStage<DS, NB * 8>::BYTES, 80 * 1024);
    cudaFuncSetAttribute(matvec32u_kernel<DS, NB, KER, UH>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         smem);
    dim3 g((unsigned)((n + UR - 1) / UR), (unsigned)js);
    matvec32u_kernel<DS, NB, KER, UH><<<g, umma_threads(UH), smem, s>>>(Xs, n, Xpr, Pk, part, chunk_st,
                                                                         nstage, err, wait_limit_ns());
}

// the tcgen05 matvec with the row-warp split UH picked by the autotuner
// (1 or 2 row warps per TMEM lane quarter; both form every kernel value and
// column sum identically, so the choice never changes a result)
template <int DS, int NB, int KER>
static void launch_u_any(const float *Xs, int64_t n, float *Xpr, const uint32_t *Pk, float *part,
                         int js, int64_t chunk_st, int64_t npad, int *err, cudaStream_t s)
{
    const int64_t nst = npad / UJ;
    const unsigned gb = (unsigned)((npad + 255) / 256);
    upoints_kernel<<<gb, 256, 0, s>>>(Xs, n, DS, npad, Xpr);
    char key[96];
    snprintf(key, sizeof(key), "mv32u/ds%d/nb%d/ker%d/n2^%d/%s", DS, NB, KER, log2_bucket(n),
             tune_device_tag().c_str());
    if constexpr (NB == 8) {
        // 64 columns: two row warps per lane quarter, each folding 32 columns
        launch_u<DS, NB, KER, 2>(Xs, n, Xpr, Pk, part, js, chunk_st, nst, err, s);
        return;
    } else {
        auto run = [&](int c) {
            if (c == 1) launch_u<DS, NB, KER, 2>(Xs, n, Xpr, Pk, part, js, chunk_st, nst, err, s);
            else launch_u<DS, NB, KER, 1>(Xs, n, Xpr, Pk, part, js, chunk_st, nst, err, s);
        };
        tune_run(key, 2, run, s, 0);
    }
}

// columns per launch of the FP32 matvec: 64 on the tcgen05 path (one kernel
// value feeds all 64), else at most 32
static int piece_cap(int nrhs) { return (nrhs >= 64 && nrhs % 16 == 0) ? 64 : 32; }

size_t matvec32_scratch(int64_t n, int nrhs)
{
    const int cap = piece_cap(nrhs);
    const size_t part = sizeof(float) * (size_t)std::max(pick_js(n), UJS_MAX) *
                        (size_t)std::min(std::max(nrhs, 1), cap) * (size_t)n;
    const size_t np = (size_t)tc_npad(n);
    const size_t dup = sizeof(f2_t) * np * 18;                     // DS + 2 <= 18
    // the mma.sync tile's split p rows, or the tcgen05 path's hi/lo halves of cap columns
    const size_t psp = sizeof(uint32_t) * np * (size_t)std::max(TcRow<4>::ROW, 2 * cap);
    return (part + 255) / 256 * 256 + (dup + 255) / 256 * 256 + psp + 256;
}


template <int DS, int NB, int KER>
static void launch_tca(const float *Xs, int64_t n, const f2_t *Xdup, const uint32_t *Psp,
                       float *part, int js, int64_t chunk, int *err, cudaStream_t s)
{
    const int smem = 2 * TcStage<DS, NB>::BYTES;
    cudaFuncSetAttribute(matvec32tca_kernel<DS, NB, KER>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    dim3 g((unsigned)((n + TCR - 1) / TCR), (unsigned)js);
    matvec32tca_kernel<DS, NB, KER><<<g, 256, smem, s>>>(Xs, n, Xdup, Psp, part, chunk, err);
}


struct TcPrep {           // prepared operands of the asynchronous TC paths
    f2_t *Xdup;              // mma.sync path: duplicated points; tcgen05 path: Xpr
    uint32_t *Psp;           // mma.sync path: Psp; tcgen05 path: Pk
    int64_t npad;
    int *err;
    bool umma;               // tcgen05 path for 16 and 32 right-hand sides
    int jsu;                 // its j-chunks
    int64_t chunk_st;
};

template <int D, int NR, int KER>
static void launch32(const float *Xs, int64_t n, const float *P, float *part, int js,
                     int64_t chunk, const TcPrep &tp, cudaStream_t s)
{
    dim3 grid((unsigned)((n + TI - 1) / TI), (unsigned)js);
    if constexpr (NR == 64) {
        // only the tcgen05 path takes 64-column pieces
        constexpr int DS = (D == 3 ? 4 : D);
        const int64_t tot = tp.npad * NR;
        ksplit_kernel<NR><<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(P, n, n, tp.npad, tp.Psp);
        launch_u_any<DS, 8, KER>(Xs, n, reinterpret_cast<float *>(tp.Xdup), tp.Psp, part, tp.jsu,
                                 tp.chunk_st, tp.npad, tp.err, s);
        return;
    } else if constexpr (NR >= 16) {
        if (tp.umma) {
            constexpr int DS = (D == 3 ? 4 : D);
            const int64_t tot = tp.npad * NR;
            ksplit_kernel<NR><<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(P, n, n, tp.npad, tp.Psp);
            launch_u_any<DS, NR / 8, KER>(Xs, n, reinterpret_cast<float *>(tp.Xdup),
                                          tp.Psp, part, tp.jsu, tp.chunk_st, tp.npad, tp.err, s);
            return;
        }
    }
    if constexpr (NR >= 8) {
        constexpr int DS = (D == 3 ? 4 : D);
        const int64_t tot = tp.npad * NR;
        psplit_kernel<NR / 8><<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(P, n, n, tp.npad, tp.Psp);
        launch_tca<DS, NR / 8, KER>(Xs, n, tp.Xdup, tp.Psp, part, js, chunk, tp.err, s);
    } else if constexpr (NR >= 2) {
        matvec32p_kernel<(D == 3 ? 4 : D), NR, KER><<<grid, NT, 0, s>>>(Xs, n, P, n, part, chunk);
    } else {
        // one right-hand side: two rows per thread
        dim3 g2((unsigned)((n + TI2 - 1) / TI2), (unsigned)js);
        matvec32r2_kernel<D, KER><<<g2, NT, 0, s>>>(Xs, n, P, part, chunk);
    }
}

template <int D, int KER>
static void launch32_nr(int nr, const float *Xs, int64_t n, const float *P, float *part, int js,
                        int64_t chunk, const TcPrep &tp, cudaStream_t s)
{
    switch (nr) {
    case 1: launch32<D, 1, KER>(Xs, n, P, part, js, chunk, tp, s); break;
    case 2: launch32<D, 2, KER>(Xs, n, P, part, js, chunk, tp, s); break;
    case 4: launch32<D, 4, KER>(Xs, n, P, part, js, chunk, tp, s); break;
    case 8: launch32<D, 8, KER>(Xs, n, P, part, js, chunk, tp, s); break;
    case 16: launch32<D, 16, KER>(Xs, n, P, part, js, chunk, tp, s); break;
    case 32: launch32<D, 32, KER>(Xs, n, P, part, js, chunk, tp, s); break;
    default: launch32<D, 64, KER>(Xs, n, P, part, js, chunk, tp, s); break;
    }
}

template <int KER>
static void launch32_d(int dp, int nr, const float *Xs, int64_t n, const float *P, float *part,
                       int js, int64_t chunk, const TcPrep &tp, cudaStream_t s)
{
    switch (dp) {
    case 3: launch32_nr<3, KER>(nr, Xs, n, P, part, js, chunk, tp, s); break;
    case 4: launch32_nr<4, KER>(nr, Xs, n, P, part, js, chunk, tp, s); break;
    case 8: launch32_nr<8, KER>(nr, Xs, n, P, part, js, chunk, tp, s); break;
    default: launch32_nr<16, KER>(nr, Xs, n, P, part, js, chunk, tp, s); break;
    }
}

// p, q: n x nrhs column-major with leading dimension n.
afn_status matvec32(const float *Xs, int64_t n, int dp, int kernel, float mu, const float *p,
                    int nrhs, float *q, void *scratch, size_t scratch_bytes, int *err,
                    cudaStream_t s)
{
    if (n <= 0 || nrhs <= 0) return AFN_OK;
    if (scratch_bytes < matvec32_scratch(n, nrhs)) {
        set_error("matvec32: scratch too small");
        return AFN_ERR_ARG;
    }
    if (nrhs >= 8 && !err) {
        set_error("matvec32: the tensor-core path needs a status word");
        return AFN_ERR_ARG;
    }
    int js;
    int64_t chunk;
    chunking(n, js, chunk);
    float *part = static_cast<float *>(scratch);
    TcPrep tp{};
    tp.npad = tc_npad(n);
    tp.err = err;
    {
        char *b = static_cast<char *>(scratch);
        const size_t pb = sizeof(float) * (size_t)std::max(js, UJS_MAX) *
                          (size_t)std::min(std::max(nrhs, 1), piece_cap(nrhs)) * (size_t)n;
        f2_t *xd = reinterpret_cast<f2_t *>(b + (pb + 255) / 256 * 256);
        const size_t db = sizeof(f2_t) * (size_t)tp.npad * 18;
        tp.Psp = reinterpret_cast<uint32_t *>(reinterpret_cast<char *>(xd) + (db + 255) / 256 * 256);
        tp.Xdup = xd;
        tp.umma = nrhs >= 16 && nrhs % 16 == 0;
        if (tp.umma) {
            chunking_u(n, tp.npad / UJ, tp.jsu, tp.chunk_st);
        } else if (nrhs >= 8) {
            const int ds = stored_dim32(dp);
            const int64_t tot = tp.npad * (ds + 2);
            dup_points_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(Xs, n, ds, tp.npad, xd);
        }
    }
    for (int c0 = 0; c0 < nrhs;) {
        int b = piece(nrhs - c0, tp.umma ? piece_cap(nrhs - c0) : 32);
        const float *pp = p + (int64_t)c0 * n;
        if (kernel == 0) launch32_d<0>(dp, b, Xs, n, pp, part, js, chunk, tp, s);
        else launch32_d<1>(dp, b, Xs, n, pp, part, js, chunk, tp, s);
        int64_t tot = n * b;
        const int jsb = (tp.umma && b >= 16) ? tp.jsu : js;
        matvec_finish<float><<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(
            part, jsb, b, n, pp, n, q + (int64_t)c0 * n, n, mu);
        c0 += b;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "matvec32 launch");
    return AFN_OK;
}

// ------------------------------------------------------------------ FP64 --
// FP64 tile: a 256-thread CTA = TI rows x JG j-groups.  Each thread sums
// K(x_i, x_j) p_j over its j-group of every staged tile of [j0, j1) for row
// i = row0 + threadIdx.x % TI; the j-groups are then reduced in shared memory
// in a fixed order, and on return threads with threadIdx.x < TI hold the
// row's sums in acc.  sm holds max(TJ*D + NR*TJ, (JG-1)*TI*NR) doubles.
template <int D, int NR>
struct Mv64Smem {
    static constexpr int TILE = TJ * D + NR * TJ;
    static constexpr int RED = (JG - 1) * TI * NR;
    static constexpr int v = TILE > RED ? TILE : RED;
};

template <int D, int NR>
__device__ __forceinline__ void mv64_rows(const double *__restrict__ X, int d, int64_t n,
                                          int kernel, double l, const double *__restrict__ P,
                                          int64_t ldp, int64_t row0, int64_t j0, int64_t j1,
                                          double *sm, double (&acc)[NR])
{
    double *xs = sm;
    double *ps = sm + TJ * D;
    const int ti = threadIdx.x % TI;
    const int g = threadIdx.x / TI;
    const int64_t i = row0 + ti;
    double xi[D];
#pragma unroll
    for (int t = 0; t < D; ++t) xi[t] = (i < n && t < d) ? X[i * d + t] : 0.0;
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
    if (g == 0) {
#pragma unroll
        for (int c = 0; c < NR; ++c)
            for (int q = 1; q < JG; ++q) acc[c] += sm[((q - 1) * NR + c) * TI + ti];
    }
}

template <int D, int NR>
__global__ void __launch_bounds__(NT) matvec64_kernel(const double *__restrict__ X, int d,
                                                      int64_t n, int kernel, double l,
                                                      const double *__restrict__ P, int64_t ldp,
                                                      double *__restrict__ part, int64_t chunk)
{
    __shared__ double sm[Mv64Smem<D, NR>::v];
    const int64_t i = (int64_t)blockIdx.x * TI + threadIdx.x % TI;
    const int64_t j0 = (int64_t)blockIdx.y * chunk;
    const int64_t j1 = min(n, j0 + chunk);
    double acc[NR];
    mv64_rows<D, NR>(X, d, n, kernel, l, P, ldp, (int64_t)blockIdx.x * TI, j0, j1, sm, acc);
    if (threadIdx.x < TI && i < n) {
#pragma unroll
        for (int c = 0; c < NR; ++c) part[((int64_t)blockIdx.y * NR + c) * n + i] = acc[c];
    }
}

size_t matvec64_scratch(int64_t n, int nrhs)
{
    // the same scratch serves the double-float matvec of mixed handles
    return std::max(sizeof(double) * (size_t)pick_js(n) * (size_t)std::min(std::max(nrhs, 1), 32) *
                        (size_t)n + 256,
                    matvecdf_scratch(n, nrhs));
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

// ----------------------------------------------------- double-float --
// FP64-accurate matvec for the residual replacements of the mixed solve,
// computed in double-float on the FP32 pipes (matvec_df.cuh).  Same CTA
// shape and split-K partials as the FP64 kernel: TI rows x JG j-groups,
// TJ-point tiles of the prescaled double-float points and of p (split into
// double-float) in shared memory, partial sums per j-chunk in FP64.
__device__ __forceinline__ void df_table_init(DfExpTable &T)
{
    if (threadIdx.x < 64) {
        const double v = exp2((double)threadIdx.x / 64.0);
        const float h = (float)v;
        T.t_h[threadIdx.x] = h;
        T.t_l[threadIdx.x] = (float)(v - (double)h);
    }
    if (threadIdx.x == 64) {
        const double ln2 = 0.6931471805599453094, log2e = 1.4426950408889634074;
        T.ln2_h = (float)ln2;
        T.ln2_l = (float)(ln2 - (double)T.ln2_h);
        T.log2e_h = (float)log2e;
        T.log2e_l = (float)(log2e - (double)T.log2e_h);
    }
}

}  // namespace afn
#include "matvec_dfu.cuh"
namespace afn {

template <int DS, int NR>
struct MvDfSmem {
    static constexpr int TILE = TJ * DS * 2 + NR * TJ * 2;   // floats
    static constexpr int RED = (JG - 1) * TI * NR * 2;       // floats (doubles x 2)
    static constexpr int v = TILE > RED ? TILE : RED;
};

// On return threads with threadIdx.x < TI hold row (row0 + threadIdx.x)'s
// sums over [j0, j1) in acc.
template <int DS, int NR, int KER>
__device__ __forceinline__ void mvdf_rows(const float2 *__restrict__ Xd, int64_t n,
                                          const double *__restrict__ P, int64_t ldp,
                                          int64_t row0, int64_t j0, int64_t j1, float *sm,
                                          const DfExpTable &T, double (&acc)[NR])
{
    float2 *xs = reinterpret_cast<float2 *>(sm);
    float2 *ps = xs + TJ * DS;
    const int ti = threadIdx.x % TI;
    const int g = threadIdx.x / TI;
    const int64_t i = row0 + ti;
    dfl xi[DS];
#pragma unroll
    for (int q = 0; q < DS; ++q) {
        const float2 v = i < n ? Xd[i * DS + q] : make_float2(0.f, 0.f);
        xi[q] = dfl{v.x, v.y};
    }
    float S[NR], Cc[NR];
#pragma unroll
    for (int c = 0; c < NR; ++c) S[c] = Cc[c] = 0.f;
    // the point tile holds packed pairs: points 2m, 2m + 1 and dimension q at
    // float4 m DS + q = {h, h', l, l'} (two kernel values per f32x2 operation)
    float *xsf = reinterpret_cast<float *>(xs);
    const float4 *xs4 = reinterpret_cast<const float4 *>(xs);
    for (int64_t jt = j0; jt < j1; jt += TJ) {
        __syncthreads();
        for (int e = threadIdx.x; e < TJ * DS; e += NT) {
            const int jj = e / DS, q = e % DS;
            const int64_t j = jt + jj;
            const float2 v = j < j1 ? Xd[jt * DS + e] : make_float2(0.f, 0.f);
            float *b = xsf + ((jj >> 1) * DS + q) * 4;
            b[jj & 1] = v.x;
            b[2 + (jj & 1)] = v.y;
        }
        for (int e = threadIdx.x; e < NR * TJ; e += NT) {
            const int c = e / TJ, jj = e % TJ;
            const int64_t j = jt + jj;
            const double v = j < j1 ? P[c * ldp + j] : 0.0;
            const float h = (float)v;
            ps[e] = make_float2(h, (float)(v - (double)h));
        }
        __syncthreads();
        for (int jj = g * (TJ / JG); jj < (g + 1) * (TJ / JG); jj += 2) {
            // kernel values of points jj and jj + 1 together, then their terms in order
            const dfl2 kv2 = df_kernel2<KER>(df_dist2_2<DS>(xi, xs4 + (jj >> 1) * DS), T);
            dfl kvs[2];
            f2_unpack(kv2.h, kvs[0].h, kvs[1].h);
            f2_unpack(kv2.l, kvs[0].l, kvs[1].l);
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const dfl kv = kvs[u];
#pragma unroll
                for (int c = 0; c < NR; ++c) {
                    const float2 x = ps[c * TJ + jj + u];
                    const float p = __fmul_rn(kv.h, x.x);
                    float e = __fmaf_rn(kv.h, x.x, -p);
                    e = __fmaf_rn(kv.h, x.y, e);
                    e = __fmaf_rn(kv.l, x.x, e);
                    float t;
                    two_sum(S[c], p, S[c], t);
                    Cc[c] = __fadd_rn(Cc[c], __fadd_rn(t, e));
                }
            }
        }
        // renormalise so the correction term stays small next to the sum
#pragma unroll
        for (int c = 0; c < NR; ++c) {
            float h, l;
            two_sum(S[c], Cc[c], h, l);
            S[c] = h;
            Cc[c] = l;
        }
    }
#pragma unroll
    for (int c = 0; c < NR; ++c) acc[c] = (double)S[c] + (double)Cc[c];
    __syncthreads();
    double *red = reinterpret_cast<double *>(sm);
    if (g > 0) {
#pragma unroll
        for (int c = 0; c < NR; ++c) red[((g - 1) * NR + c) * TI + ti] = acc[c];
    }
    __syncthreads();
    if (g == 0) {
#pragma unroll
        for (int c = 0; c < NR; ++c)
            for (int q = 1; q < JG; ++q) acc[c] += red[((q - 1) * NR + c) * TI + ti];
    }
}

template <int DS, int NR, int KER>
__global__ void __launch_bounds__(NT) matvecdf_kernel(const float2 *__restrict__ Xd, int64_t n,
                                                      const double *__restrict__ P, int64_t ldp,
                                                      double *__restrict__ part, int64_t chunk,
                                                      int js)
{
    extern __shared__ __align__(16) float dfsm[];   // MvDfSmem<DS, NR>::v floats
    float *sm = dfsm;
    __shared__ DfExpTable T;
    df_table_init(T);
    // tiles (row tile, j-chunk), one per CTA or -- with a capped grid -- a
    // grid-stride loop over them
    const int64_t rt = (n + TI - 1) / TI;
    const int64_t ntiles = rt * js;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t rb = tile % rt, q = tile / rt;
        const int64_t i = rb * TI + threadIdx.x % TI;
        const int64_t j0 = q * chunk;
        const int64_t j1 = min(n, j0 + chunk);
        double acc[NR];
        mvdf_rows<DS, NR, KER>(Xd, n, P, ldp, rb * TI, j0, j1, sm, T, acc);
        if (threadIdx.x < TI && i < n) {
#pragma unroll
            for (int c = 0; c < NR; ++c) part[(q * NR + c) * n + i] = acc[c];
        }
        __syncthreads();   // sm is reused by the next tile
    }
}

// fraction of the GPU a double-float matvec launched from this thread may
// occupy (CTA slots); solves running beside a group of other systems cap it
// so that the group's short kernels find free SMs
static thread_local const std::atomic<double> *tl_df_share = nullptr;
GridShareGuard::GridShareGuard(const std::atomic<double> *share) : prev(tl_df_share)
{
    tl_df_share = share;
}
GridShareGuard::~GridShareGuard() { tl_df_share = prev; }

template <int DS, int KER>
static void launchdf_nr(int nr, const float2 *Xd, int64_t n, const double *P, double *part,
                        int js, int64_t chunk, cudaStream_t s)
{
    const int64_t ntiles = (n + TI - 1) / TI * js;
    int64_t g = ntiles;
    const double share = tl_df_share ? tl_df_share->load(std::memory_order_relaxed) : 1.0;
    if (share < 1.0) g = std::min<int64_t>(g, persistent_grid(2, share));
    const unsigned grid = (unsigned)g;
    auto go = [&](auto nrc) {
        constexpr int NR = decltype(nrc)::value;
        const int smem = (int)(sizeof(float) * MvDfSmem<DS, NR>::v);
        cudaFuncSetAttribute(matvecdf_kernel<DS, NR, KER>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        matvecdf_kernel<DS, NR, KER><<<grid, NT, smem, s>>>(Xd, n, P, n, part, chunk, js);
    };
    switch (nr) {
    case 1: go(std::integral_constant<int, 1>{}); break;
    case 2: go(std::integral_constant<int, 2>{}); break;
    case 4: go(std::integral_constant<int, 4>{}); break;
    case 8: go(std::integral_constant<int, 8>{}); break;
    case 16: go(std::integral_constant<int, 16>{}); break;
    default: go(std::integral_constant<int, 32>{}); break;
    }
}

static constexpr int DUJS_MAX = 8;   // j-chunks of the tcgen05 double-float path

// scratch of the tcgen05 double-float matvec: partials (up to DUJS_MAX chunks
// x 32 columns, FP64), the digit tiles of p, the staged points, column maxima
// and exponents
static size_t dfu_scratch(int64_t n)
{
    const size_t np = (size_t)((n + DU_J - 1) / DU_J * DU_J);
    const size_t part = sizeof(double) * (size_t)DUJS_MAX * DU_NR * (size_t)n;
    const size_t dig = 2 * np * (size_t)(DU_DIG * DU_NR);
    const size_t pts = sizeof(float2) * np * 16;
    return (part + 255) / 256 * 256 + (dig + 255) / 256 * 256 + (pts + 255) / 256 * 256 + 1024;
}

static bool df_on_tc(int64_t n, int nrhs, int sum)
{
    return sum == DF_SUM_TC || (sum == DF_SUM_AUTO && use_dfu(n, nrhs));
}

size_t matvecdf_scratch(int64_t n, int nrhs, int sum)
{
    const size_t cuda_core = sizeof(double) * (size_t)pick_js(n) *
                                 (size_t)std::min(std::max(nrhs, 1), 32) * (size_t)n + 256;
    return std::max(cuda_core, df_on_tc(n, nrhs, sum) ? dfu_scratch(n) : (size_t)0);
}

size_t matvecdf_scratch(int64_t n, int nrhs) { return matvecdf_scratch(n, nrhs, DF_SUM_AUTO); }

// the double-float matvec in column pieces of at most cap (16 or 32): every
// column's sum is formed the same way whatever the piece, so the results do
// not depend on cap
static void matvec_df_pieces(int cap, const float2 *Xd, int64_t n, int ds, int kernel, double mu,
                             const double *p, int nrhs, double *q, double *part, int js,
                             int64_t chunk, cudaStream_t s)
{
    for (int c0 = 0; c0 < nrhs;) {
        const int b = piece(nrhs - c0, cap);
        const double *pp = p + (int64_t)c0 * n;
        const int key = ds * 2 + kernel;
        switch (key) {
        case 8: launchdf_nr<4, 0>(b, Xd, n, pp, part, js, chunk, s); break;
        case 9: launchdf_nr<4, 1>(b, Xd, n, pp, part, js, chunk, s); break;
        case 16: launchdf_nr<8, 0>(b, Xd, n, pp, part, js, chunk, s); break;
        case 17: launchdf_nr<8, 1>(b, Xd, n, pp, part, js, chunk, s); break;
        case 32: launchdf_nr<16, 0>(b, Xd, n, pp, part, js, chunk, s); break;
        default: launchdf_nr<16, 1>(b, Xd, n, pp, part, js, chunk, s); break;
        }
        const int64_t tot = n * b;
        matvec_finish<double><<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(
            part, js, b, n, pp, n, q + (int64_t)c0 * n, n, mu);
        c0 += b;
    }
}

// ------------------------------------ double-float on the tensor cores --
// the double-float points for the staged tiles, zero-padded, as packed pairs:
// points 2m, 2m + 1 and dimension q at float4 m ds + q = {h, h', l, l'}
__global__ void dupoints_kernel(const float2 *__restrict__ Xd, int64_t n, int ds, int64_t npad,
                                float4 *__restrict__ Xpr)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= npad / 2 * ds) return;
    const int64_t m = e / ds;
    const int q = (int)(e % ds);
    const int64_t j0 = 2 * m, j1 = 2 * m + 1;
    const float2 a = j0 < n ? Xd[j0 * ds + q] : make_float2(0.f, 0.f);
    const float2 b = j1 < n ? Xd[j1 * ds + q] : make_float2(0.f, 0.f);
    Xpr[e] = make_float4(a.x, b.x, a.y, b.y);
}

// max_j |p_jc| of the nc columns, as the bits of a non-negative double
__global__ void du_colmax_kernel(const double *__restrict__ p, int64_t n, int nc,
                                 unsigned long long *__restrict__ mx)
{
    const int c = blockIdx.y;
    double m = 0.0;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n;
         j += (int64_t)gridDim.x * blockDim.x)
        m = fmax(m, fabs(p[(int64_t)c * n + j]));
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0 && m > 0.0)
        atomicMax(mx + c, (unsigned long long)__double_as_longlong(m));
}

// the digit tiles of p: with 2^E > max_j |p_jc| (frexp), p_jc 2^(7-E) = sum_t
// b_t 2^(-8t), each digit the nearest integer of the remainder so far (every
// step exact in FP64); one thread per (stage, column, point)
__global__ void du_pdigits_kernel(const double *__restrict__ p, int64_t n, int nc, int64_t npad,
                                  const unsigned long long *__restrict__ mx, int *__restrict__ pexp,
                                  __nv_bfloat16 *__restrict__ Pd)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= npad * DU_NR) return;
    const int kk = (int)(e % DU_J);
    const int c = (int)((e / DU_J) % DU_NR);
    const int64_t st = e / (DU_J * DU_NR);
    const int64_t j = st * DU_J + kk;
    int E = 0;
    double w = 0.0;
    if (c < nc) {
        const double m = __longlong_as_double((long long)mx[c]);
        if (m > 0.0) frexp(m, &E);
        if (j == 0) pexp[c] = E;
        if (j < n) w = ldexp(p[(int64_t)c * n + j], 7 - E);
    }
    __nv_bfloat16 *tile = Pd + st * (int64_t)(DU_J * DU_DIG * DU_NR);
#pragma unroll
    for (int t = 0; t < DU_DIG; ++t) {
        const double d = rint(w);
        w = (w - d) * 256.0;
        tile[du_tile_elem(t * DU_NR + c, kk)] = __double2bfloat16(d);
    }
}

// j-chunks (in staged tiles) of the tcgen05 double-float path: the count whose
// CTAs (one per SM) fill the last wave best, chunks of at least 8 tiles
static void chunking_du(int64_t n, int64_t nstage, int &js, int64_t &chunk_st)
{
    const int64_t rt = (n + UR - 1) / UR;
    const int64_t slots = num_sms();
    double best = -1.0;
    js = 1;
    chunk_st = nstage;
    for (int q = 1; q <= DUJS_MAX; ++q) {
        const int64_t cs = (nstage + q - 1) / q;
        if (q > 1 && cs < 8) break;
        const int64_t jq = (nstage + cs - 1) / cs;
        const int64_t tot = rt * jq;
        const int64_t waves = (tot + slots - 1) / slots;
        const double eff = (double)tot / (double)(waves * slots);
        if (eff > best + 1e-9) {
            best = eff;
            js = (int)jq;
            chunk_st = cs;
        }
    }
}

template <int DS, int KER>
static void launch_du(const float2 *Xd, int64_t n, const float2 *Xpr, const __nv_bfloat16 *Pd,
                      const int *pexp, double *part, int nc, int js, int64_t chunk_st,
                      int64_t nstage, int *err, cudaStream_t s)
{
    constexpr int smem = DuStage<DS>::SMEM;
    cudaFuncSetAttribute(matvecdfu_kernel<DS, KER>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    dim3 g((unsigned)((n + UR - 1) / UR), (unsigned)js);
    matvecdfu_kernel<DS, KER><<<g, DU_THREADS, smem, s>>>(Xd, n, Xpr, Pd, pexp, part, nc, chunk_st,
                                                          nstage, err, wait_limit_ns());
}

// the double-float matvec with the contraction on the tensor cores, in pieces
// of 32 columns (the last one zero-padded)
static afn_status matvec_dfu(const float2 *Xd, int64_t n, int ds, int kernel, double mu,
                             const double *p, int nrhs, double *q, void *scratch, int *err,
                             cudaStream_t s)
{
    const int64_t npad = (n + DU_J - 1) / DU_J * DU_J, nstage = npad / DU_J;
    char *c = static_cast<char *>(scratch);
    double *part = reinterpret_cast<double *>(c);
    c += (sizeof(double) * (size_t)DUJS_MAX * DU_NR * (size_t)n + 255) / 256 * 256;
    __nv_bfloat16 *Pd = reinterpret_cast<__nv_bfloat16 *>(c);
    c += (2 * (size_t)npad * (DU_DIG * DU_NR) + 255) / 256 * 256;
    float2 *Xpr = reinterpret_cast<float2 *>(c);
    c += (sizeof(float2) * (size_t)npad * 16 + 255) / 256 * 256;
    unsigned long long *mx = reinterpret_cast<unsigned long long *>(c);
    int *pexp = reinterpret_cast<int *>(c + 512);
    int js;
    int64_t chunk_st;
    chunking_du(n, nstage, js, chunk_st);
    dupoints_kernel<<<(unsigned)((npad / 2 * ds + 255) / 256), 256, 0, s>>>(
        Xd, n, ds, npad, reinterpret_cast<float4 *>(Xpr));
    for (int c0 = 0; c0 < nrhs; c0 += DU_NR) {
        const int nc = std::min(DU_NR, nrhs - c0);
        const double *pp = p + (int64_t)c0 * n;
        AFN_CUDA(cudaMemsetAsync(mx, 0, sizeof(unsigned long long) * DU_NR, s));
        du_colmax_kernel<<<dim3((unsigned)std::min<int64_t>((n + 255) / 256, 256), (unsigned)nc), 256, 0, s>>>(
            pp, n, nc, mx);
        du_pdigits_kernel<<<(unsigned)((npad * DU_NR + 255) / 256), 256, 0, s>>>(pp, n, nc, npad, mx,
                                                                                 pexp, Pd);
        switch (ds * 2 + kernel) {
        case 8: launch_du<4, 0>(Xd, n, Xpr, Pd, pexp, part, nc, js, chunk_st, nstage, err, s); break;
        case 9: launch_du<4, 1>(Xd, n, Xpr, Pd, pexp, part, nc, js, chunk_st, nstage, err, s); break;
        case 16: launch_du<8, 0>(Xd, n, Xpr, Pd, pexp, part, nc, js, chunk_st, nstage, err, s); break;
        case 17: launch_du<8, 1>(Xd, n, Xpr, Pd, pexp, part, nc, js, chunk_st, nstage, err, s); break;
        case 32: launch_du<16, 0>(Xd, n, Xpr, Pd, pexp, part, nc, js, chunk_st, nstage, err, s); break;
        default: launch_du<16, 1>(Xd, n, Xpr, Pd, pexp, part, nc, js, chunk_st, nstage, err, s); break;
        }
        const int64_t tot = n * nc;
        matvec_finish<double><<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(
            part, js, nc, n, pp, n, q + (int64_t)c0 * n, n, mu);
    }
    return AFN_OK;
}

afn_status matvec_df(const float2 *Xd, int64_t n, int ds, int kernel, double mu, const double *p,
                     int nrhs, double *q, void *scratch, size_t scratch_bytes, int *err,
                     cudaStream_t s, int sum)
{
    if (n <= 0 || nrhs <= 0) return AFN_OK;
    if (scratch_bytes < matvecdf_scratch(n, nrhs, sum)) {
        set_error("matvec_df: scratch too small");
        return AFN_ERR_ARG;
    }
    if (df_on_tc(n, nrhs, sum)) {
        // the contraction on the tensor cores
        AFN_TRY(matvec_dfu(Xd, n, ds, kernel, mu, p, nrhs, q, scratch, err, s));
    } else {
        int js;
        int64_t chunk;
        chunking(n, js, chunk);
        matvec_df_pieces(16, Xd, n, ds, kernel, mu, p, nrhs, q, static_cast<double *>(scratch), js,
                         chunk, s);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "matvec_df launch");
    return AFN_OK;
}

// double-float prescaled points: x * scale as (hi, lo) floats, n x ds
__global__ void points_df_kernel(const double *__restrict__ X, int64_t n, int d, int ds,
                                 double scale, float2 *__restrict__ Xd)
{
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n * ds) return;
    const int64_t i = e / ds;
    const int t = (int)(e % ds);
    const double v = t < d ? X[i * d + t] * scale : 0.0;
    const float h = (float)v;
    Xd[e] = make_float2(h, (float)(v - (double)h));
}

afn_status make_points_df(const double *X, int64_t n, int d, int ds, int kernel, double l,
                          float2 *Xd, cudaStream_t s)
{
    const double scale = (kernel == 0) ? 1.2011224087864498 / l    // sqrt(log2 e) / l
                                       : 1.7320508075688772 / l;   // sqrt(3) / l
    const int64_t tot = n * ds;
    if (tot == 0) return AFN_OK;
    points_df_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(X, n, d, ds, scale, Xd);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "points_df launch");
    return AFN_OK;
}

// ----------------------------------------------- row sums of the kernel --
__global__ void fill_ones_kernel(float *p, int64_t n)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = 1.f;
}

__global__ void max_kernel(const float *q, int64_t n, unsigned int *out)
{
    float m = 0.f;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        m = fmaxf(m, q[i]);
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, __float_as_uint(m));   // m >= 0
}

afn_status kernel_row_sum_max(const float *Xs, int64_t n, int dp, int kernel, double *out,
                              cudaStream_t s)
{
    DevBuf buf, scratch;
    const size_t sb = matvec32_scratch(n, 1);
    AFN_TRY(buf.alloc(sizeof(float) * 2 * (size_t)n + 256));
    AFN_TRY(scratch.alloc(sb));
    float *p = buf.as<float>(), *q = p + n;
    unsigned int *mx = reinterpret_cast<unsigned int *>(q + n);
    fill_ones_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(p, n);
    AFN_TRY(matvec32(Xs, n, dp, kernel, 0.f, p, 1, q, scratch.p, sb, nullptr, s));   // 1 column: no TC
    AFN_CUDA(cudaMemsetAsync(mx, 0, sizeof(unsigned int), s));
    max_kernel<<<(unsigned)std::min<int64_t>((n + 255) / 256, 1024), 256, 0, s>>>(q, n, mx);
    unsigned int bits = 0;
    AFN_CUDA(cudaMemcpyAsync(&bits, mx, sizeof(bits), cudaMemcpyDeviceToHost, s));
    AFN_CUDA(cudaStreamSynchronize(s));
    float v;
    memcpy(&v, &bits, sizeof(v));
    *out = (double)v;
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

// ------------------------------------------------------ grouped matvecs --
// One persistent launch over the 128-row (FP32) or 64-row (FP64) tiles of
// every member system of a group.  A tile covers one column group of 8
// right-hand sides and the whole j range of its system, so each output
// element is summed by one CTA in a fixed order and a system's result does
// not depend on which other systems share the launch.

__device__ __forceinline__ bool group_live(const GSys &S, int cg)
{
    const int c0 = cg * GC, c1 = min(S.nrhs, c0 + GC);
    for (int c = c0; c < c1; ++c)
        if (S.cs[c].active) return true;
    return false;
}

static constexpr int GMV32_MINB = 3;

// tiles staged by bulk copies from the system's Xdup and Psp (written by the
// beta/p update), double-buffered; the mbarriers persist over the CTA's tiles
__global__ void __launch_bounds__(256, GMV32_MINB) gmv32_kernel(const GDev *__restrict__ gd)
{
    __shared__ __align__(16) unsigned char stage[2 * TcStage<16, 1>::BYTES];
    __shared__ __align__(8) uint64_t bars[2];
    if (threadIdx.x == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        mbar_init_fence();
    }
    __syncthreads();
    uint32_t parity = 0;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = lane >> 2, t = lane & 3;
    const int nt = gd->nmv;
    for (int ti = blockIdx.x; ti < nt; ti += gridDim.x) {
        const GTile tl = gd->mv[ti];
        const GSys &S = gd->sys[tl.sys];
        if (!group_live(S, tl.cg)) continue;
        const int64_t n = S.n;
        const f2_t *xd = reinterpret_cast<const f2_t *>(S.Xdup);
        const uint32_t *ps = S.Psp + (int64_t)tl.cg * S.npad * TcRow<1>::ROW;
        float acc[1][4];
        bool ok;
        switch (S.ds * 2 + S.kernel) {
        case 8:  ok = mv32tc_rows_async<4, 1, 0>(S.X32, n, xd, ps, tl.r0, 0, n, stage, bars, parity, acc); break;
        case 9:  ok = mv32tc_rows_async<4, 1, 1>(S.X32, n, xd, ps, tl.r0, 0, n, stage, bars, parity, acc); break;
        case 16: ok = mv32tc_rows_async<8, 1, 0>(S.X32, n, xd, ps, tl.r0, 0, n, stage, bars, parity, acc); break;
        case 17: ok = mv32tc_rows_async<8, 1, 1>(S.X32, n, xd, ps, tl.r0, 0, n, stage, bars, parity, acc); break;
        case 32: ok = mv32tc_rows_async<16, 1, 0>(S.X32, n, xd, ps, tl.r0, 0, n, stage, bars, parity, acc); break;
        default: ok = mv32tc_rows_async<16, 1, 1>(S.X32, n, xd, ps, tl.r0, 0, n, stage, bars, parity, acc); break;
        }
        if (!ok) {
            if (threadIdx.x == 0) atomicExch(gd->err, DEV_TIMEOUT);
            return;
        }
        const int64_t ia = tl.r0 + warp * 16 + g, ib = ia + 8;
        const float mu = S.mu32;
        const float *P = S.p32 + (int64_t)tl.cg * GC * n;
        const float *p0 = P + (int64_t)(2 * t) * n, *p1 = p0 + n;
        float *q0 = S.q32 + ((int64_t)tl.cg * GC + 2 * t) * n, *q1 = q0 + n;
        if (ia < n) { q0[ia] = acc[0][0] + mu * p0[ia]; q1[ia] = acc[0][1] + mu * p1[ia]; }
        if (ib < n) { q0[ib] = acc[0][2] + mu * p0[ib]; q1[ib] = acc[0][3] + mu * p1[ib]; }
    }
}

int group_npad(int64_t n) { return (int)tc_npad(n); }

void dup_points(const float *Xs, int64_t n, int ds, int64_t npad, void *Xdup, cudaStream_t s)
{
    const int64_t tot = npad * (ds + 2);
    if (tot > 0)
        dup_points_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(Xs, n, ds, npad,
                                                                       static_cast<f2_t *>(Xdup));
}

// q = (K + mu I) x, FP64-accurate (double-float, matvec_df.cuh), for the
// systems whose residual is being replaced
__global__ void __launch_bounds__(NT) gmvdf_kernel(const GDev *__restrict__ gd)
{
    __shared__ __align__(16) float sm[MvDfSmem<16, GC>::v];
    __shared__ DfExpTable T;
    df_table_init(T);
    const int nt = gd->nmv64;
    for (int ti = blockIdx.x; ti < nt; ti += gridDim.x) {
        const GTile tl = gd->mv64[ti];
        if (!gd->rep[tl.sys]) continue;
        const GSys &S = gd->sys[tl.sys];
        const int64_t n = S.n;
        const double *P = S.x + (int64_t)tl.cg * GC * n;
        double acc[GC];
        switch (S.ds * 2 + S.kernel) {
        case 8:  mvdf_rows<4, GC, 0>(S.Xdf, n, P, n, tl.r0, 0, n, sm, T, acc); break;
        case 9:  mvdf_rows<4, GC, 1>(S.Xdf, n, P, n, tl.r0, 0, n, sm, T, acc); break;
        case 16: mvdf_rows<8, GC, 0>(S.Xdf, n, P, n, tl.r0, 0, n, sm, T, acc); break;
        case 17: mvdf_rows<8, GC, 1>(S.Xdf, n, P, n, tl.r0, 0, n, sm, T, acc); break;
        case 32: mvdf_rows<16, GC, 0>(S.Xdf, n, P, n, tl.r0, 0, n, sm, T, acc); break;
        default: mvdf_rows<16, GC, 1>(S.Xdf, n, P, n, tl.r0, 0, n, sm, T, acc); break;
        }
        const int64_t i = tl.r0 + threadIdx.x;
        if (threadIdx.x < TI && i < n) {
            double *q = S.q + (int64_t)tl.cg * GC * n;
#pragma unroll
            for (int c = 0; c < GC; ++c) q[c * n + i] = acc[c] + S.mu * P[c * n + i];
        }
    }
}

int group_mv32_rows() { return TCR; }
int group_mv64_rows() { return TI; }

int persistent_grid(int ctas_per_sm, double share)
{
    const int g = (int)(num_sms() * ctas_per_sm * share + 0.5);
    return g > 0 ? g : 1;
}

afn_status group_matvec32(const GDev *gd, cudaStream_t s, double share, int cps)
{
    gmv32_kernel<<<persistent_grid(cps > 0 ? cps : GMV32_MINB, share), 256, 0, s>>>(gd);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? AFN_OK : cuda_fail(e, "grouped matvec32 launch");
}

afn_status group_matvec64(const GDev *gd, cudaStream_t s, double share)
{
    gmvdf_kernel<<<persistent_grid(2, share), NT, 0, s>>>(gd);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? AFN_OK : cuda_fail(e, "grouped matvec64 launch");
}

}  // namespace afn
