// fsai.cu -- FSAI of the Schur complement (Alg. 1 applied as in Alg. 2):
// for every Schur row i with pattern s (its w-1 nearest lower neighbours,
// then i):
//   A = K22[s,s] + mu I - W[:,s]^T W[:,s]        (W = L^{-1} K12, Sec. 3.2)
//   y = A^{-1} e_last,  G[i,s] = y^T / sqrt(y_last)
// One launch; one CTA per row.  The Gram W[:,s]^T W[:,s] streams the
// pattern's W columns (rows of W^T, contiguous) through shared memory in
// chunks of KC landmarks; the local Cholesky and the two triangular solves
// run in shared memory in FP64.
#include <algorithm>
#include <cmath>
#include <type_traits>

#include "afn_device.cuh"
#include "afn_internal.cuh"

namespace afn {

static constexpr int KC = 32;    // landmarks per Gram chunk

// FT threads per CTA (autotuned: 128 or 256 for w <= 64, 256 or 512 above;
// every Gram entry and Cholesky step is the same sum whatever FT is).
// GDF (FP64 W only): the Gram in double-float arithmetic on the FP32 pipes,
// each staged W value split into hi + lo floats, each term by the FMA-based
// TwoProduct and the sums double-float (about 48-bit accuracy, for the
// double-float handles; GB300's FP64 pipe is far slower).
template <int WM, class TW, int FT, bool GDF>
__global__ void __launch_bounds__(FT) fsai_kernel(const double *__restrict__ Xr, int d, int kernel,
                                                  double l, double mu,
                                                  const TW *__restrict__ Wt, int64_t k,
                                                  const int32_t *__restrict__ pat, int w,
                                                  double *__restrict__ G, int *status)
{
    static_assert(!GDF || sizeof(TW) == 8, "the double-float Gram takes FP64 W");
    using WS = std::conditional_t<GDF, float2, TW>;             // staged W value
    extern __shared__ __align__(16) unsigned char smraw[];
    double *A = reinterpret_cast<double *>(smraw);              // WM x (WM+1)
    WS *ws = reinterpret_cast<WS *>(A + WM * (WM + 1));          // WM x (KC+1)
    __shared__ int32_t s[WM];
    __shared__ int m_s;
    __shared__ double piv;
    __shared__ int bad;
    const int64_t i = blockIdx.x;
    const int tid = threadIdx.x;
    if (tid == 0) {
        int m = 0;
        while (m < w && pat[i * w + m] >= 0) ++m;
        m_s = m;
        bad = 0;
    }
    if (tid < w && tid < WM) s[tid] = pat[i * w + tid];
    __syncthreads();
    const int m = m_s;
    // Gram, lower triangle, in 4 x 4 tiles: each thread a strided set of tile
    // pairs (ta >= tb), 16 sums per pair so that each staged value feeds four
    // products; every entry is still the sum over the landmarks in order
    constexpr int NTL = WM / 4;
    constexpr int MAXT = (NTL * (NTL + 1) / 2 + FT - 1) / FT;
    const int nt = (m + 3) / 4;
    const int ntt = nt * (nt + 1) / 2;
    TW acc[GDF ? 1 : MAXT][4][4];                 // the Gram in TW
    float acch[GDF ? MAXT : 1][4][4], accl[GDF ? MAXT : 1][4][4];   // or in double-float
    int ta[MAXT], tb[MAXT];
#pragma unroll
    for (int q = 0; q < MAXT; ++q) {
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                if constexpr (GDF) acch[q][r][c] = accl[q][r][c] = 0.f;
                else acc[q][r][c] = 0;
            }
        const int p = tid + q * FT;
        int a = 0, b = 0;
        if (p < ntt) {
            // p -> (a, b) with a >= b, row-major over the lower triangle of tiles
            a = (int)((sqrt(8.0 * p + 1.0) - 1.0) * 0.5);
            while ((a + 1) * (a + 2) / 2 <= p) ++a;
            while (a * (a + 1) / 2 > p) --a;
            b = p - a * (a + 1) / 2;
        }
        ta[q] = a;
        tb[q] = b;
    }
    for (int64_t k0 = 0; k0 < k; k0 += KC) {
        __syncthreads();
        // rows m .. 4 nt - 1 of the tiles are zero
        for (int e = tid; e < 4 * nt * KC; e += FT) {
            int a = e / KC, kk = e % KC;
            int64_t gk = k0 + kk;
            const TW v = (a < m && gk < k) ? Wt[(int64_t)s[a] * k + gk] : (TW)0;
            if constexpr (GDF) {
                const float h = (float)v;
                ws[a * (KC + 1) + kk] = make_float2(h, (float)((double)v - (double)h));
            } else {
                ws[a * (KC + 1) + kk] = v;
            }
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < MAXT; ++q) {
            if (tid + q * FT < ntt) {
                const WS *wa = ws + 4 * ta[q] * (KC + 1);
                const WS *wb = ws + 4 * tb[q] * (KC + 1);
#pragma unroll 4
                for (int kk = 0; kk < KC; ++kk) {
                    WS va[4], vb[4];
#pragma unroll
                    for (int r = 0; r < 4; ++r) {
                        va[r] = wa[r * (KC + 1) + kk];
                        vb[r] = wb[r * (KC + 1) + kk];
                    }
#pragma unroll
                    for (int r = 0; r < 4; ++r)
#pragma unroll
                        for (int c = 0; c < 4; ++c) {
                            if constexpr (GDF) {
                                const float p = __fmul_rn(va[r].x, vb[c].x);
                                float e = __fmaf_rn(va[r].x, vb[c].x, -p);
                                e = __fmaf_rn(va[r].x, vb[c].y, e);
                                e = __fmaf_rn(va[r].y, vb[c].x, e);
                                const float sh = acch[q][r][c];
                                const float s1 = __fadd_rn(sh, p);
                                const float bb = __fsub_rn(s1, sh);
                                const float er = __fadd_rn(__fsub_rn(sh, __fsub_rn(s1, bb)), __fsub_rn(p, bb));
                                acch[q][r][c] = s1;
                                accl[q][r][c] = __fadd_rn(accl[q][r][c], __fadd_rn(er, e));
                            } else {
                                acc[q][r][c] += va[r] * vb[c];
                            }
                        }
                }
            }
        }
    }
    // A = K22[s,s] + mu I - Gram  (lower triangle)
#pragma unroll
    for (int q = 0; q < MAXT; ++q) {
        if (tid + q * FT < ntt) {
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const int a = 4 * ta[q] + r, b = 4 * tb[q] + c;
                    if (a < m && b <= a) {
                        double r2 = sqdist_exact(Xr + (int64_t)s[a] * d, Xr + (int64_t)s[b] * d, d);
                        double v = kernel64(r2, kernel, l);
                        if (a == b) v += mu;
                        double gram;
                        if constexpr (GDF) gram = (double)acch[q][r][c] + (double)accl[q][r][c];
                        else gram = (double)acc[q][r][c];
                        A[a * (WM + 1) + b] = v - gram;
                    }
                }
        }
    }
    __syncthreads();
    // Cholesky A = R R^T in place (lower)
    for (int j = 0; j < m; ++j) {
        if (tid == 0) {
            double v = A[j * (WM + 1) + j];
            if (!(v > 0.0)) { bad = 1; v = 1.0; }
            piv = sqrt(v);
            A[j * (WM + 1) + j] = piv;
        }
        __syncthreads();
        for (int r = j + 1 + tid; r < m; r += FT) A[r * (WM + 1) + j] /= piv;
        __syncthreads();
        const int rem = m - j - 1;
        for (int e = tid; e < rem * rem; e += FT) {
            int r = j + 1 + e / rem, c = j + 1 + e % rem;
            if (c <= r) A[r * (WM + 1) + c] -= A[r * (WM + 1) + j] * A[c * (WM + 1) + j];
        }
        __syncthreads();
    }
    // R z = e_last (forward), R^T y = z (backward); y kept in ws as double
    double *y = reinterpret_cast<double *>(ws);
    if (tid < 32) {
        const int lane = tid;
        // forward substitution of e_last: z_j = 0 for j < m-1, z_last = 1 / R_last
        for (int j = lane; j < m; j += 32) y[j] = 0.0;
        __syncwarp();
        if (lane == 0) y[m - 1] = 1.0 / A[(m - 1) * (WM + 1) + m - 1];
        __syncwarp();
        for (int j = m - 1; j >= 0; --j) {
            double part = 0.0;
            for (int p = j + 1 + lane; p < m; p += 32) part += A[p * (WM + 1) + j] * y[p];
            part = warp_sum(part);
            if (lane == 0) {
                // y_j = (z_j - sum_{p>j} R_pj y_p) / R_jj  with  z = R^{-1} e_last
                double zj = (j == m - 1) ? 1.0 / A[j * (WM + 1) + j] : 0.0;
                y[j] = (zj - part) / A[j * (WM + 1) + j];
            }
            __syncwarp();
        }
        double yl = y[m - 1];
        if (!(yl > 0.0) && lane == 0) bad = 1;
        double sc = sqrt(yl > 0.0 ? yl : 1.0);
        for (int p = lane; p < w; p += 32) G[i * w + p] = (p < m) ? y[p] / sc : 0.0;
    }
    __syncthreads();
    if (tid == 0 && bad) atomicExch(status, DEV_NOT_SPD);
}

template <int WM, class TW, int FT, bool GDF>
static afn_status launch_fsai_ft(const double *Xr, int64_t nr, int d, KParams kp, const TW *Wt,
                                 int64_t k, const int32_t *pat, int w, double *G, int *status,
                                 cudaStream_t s)
{
    size_t smem = sizeof(double) * WM * (WM + 1) +
                  std::max(sizeof(TW) * WM * (KC + 1), sizeof(double) * WM);
    auto kfn = fsai_kernel<WM, TW, FT, GDF>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return cuda_fail(e, "fsai smem attribute");
    }
    for (int64_t r0 = 0; r0 < nr; r0 += 1 << 30) {
        int64_t rows = std::min<int64_t>(nr - r0, 1 << 30);
        kfn<<<(unsigned)rows, FT, smem, s>>>(Xr, d, kp.kernel, kp.l, kp.mu, Wt, k, pat + r0 * w, w,
                                             G + r0 * w, status);
    }
    AFN_CUDA(cudaGetLastError());
    return AFN_OK;
}

// the FSAI rows with the autotuned block size (each run writes the same G)
template <int WM, class TW, bool GDF>
static afn_status launch_fsai(const double *Xr, int64_t nr, int d, KParams kp, const TW *Wt,
                              int64_t k, const int32_t *pat, int w, double *G, int *status,
                              cudaStream_t s)
{
    constexpr int FA = WM <= 64 ? 128 : 256;
    char key[96];
    snprintf(key, sizeof(key), "fsai/wm%d/%s/k2^%d/nr2^%d/%s", WM,
             GDF ? "df" : sizeof(TW) == 8 ? "f64" : "f32", log2_bucket(k), log2_bucket(nr),
             tune_device_tag().c_str());
    afn_status st = AFN_OK;
    auto run = [&](int c) {
        st = c == 0 ? launch_fsai_ft<WM, TW, FA, GDF>(Xr, nr, d, kp, Wt, k, pat, w, G, status, s)
                    : launch_fsai_ft<WM, TW, 2 * FA, GDF>(Xr, nr, d, kp, Wt, k, pat, w, G, status, s);
    };
    tune_run(key, 2, run, s, 1);
    return st;
}

template <class TW, bool GDF>
static afn_status fsai_build(const double *Xr, int64_t nr, int d, KParams kp, const TW *Wt,
                             int64_t k, const int32_t *pat, int w, double *G, int *status,
                             cudaStream_t s)
{
    if (nr <= 0) return AFN_OK;
    AFN_CUDA(cudaMemsetAsync(status, 0, sizeof(int), s));
    if (w <= 32) return launch_fsai<32, TW, GDF>(Xr, nr, d, kp, Wt, k, pat, w, G, status, s);
    if (w <= 64) return launch_fsai<64, TW, GDF>(Xr, nr, d, kp, Wt, k, pat, w, G, status, s);
    if (w <= 128) return launch_fsai<128, TW, GDF>(Xr, nr, d, kp, Wt, k, pat, w, G, status, s);
    set_error("fsai: w=%d above 128 is not supported", w);
    return AFN_ERR_ARG;
}

afn_status fsai_build64(const double *Xr, int64_t nr, int d, KParams kp, const double *Wt,
                        int64_t k, const int32_t *pat, int w, double *G, int *status,
                        cudaStream_t s)
{
    return fsai_build<double, false>(Xr, nr, d, kp, Wt, k, pat, w, G, status, s);
}

afn_status fsai_build_df(const double *Xr, int64_t nr, int d, KParams kp, const double *Wt,
                         int64_t k, const int32_t *pat, int w, double *G, int *status,
                         cudaStream_t s)
{
    return fsai_build<double, true>(Xr, nr, d, kp, Wt, k, pat, w, G, status, s);
}

afn_status fsai_build32(const double *Xr, int64_t nr, int d, KParams kp, const float *Wt,
                        int64_t k, const int32_t *pat, int w, double *G, int *status,
                        cudaStream_t s)
{
    return fsai_build<float, false>(Xr, nr, d, kp, Wt, k, pat, w, G, status, s);
}

// ------------------------------------------------ CSR of G^T (gather form) --
__global__ void gt_count_kernel(const int32_t *__restrict__ pat, int64_t nnzslots,
                                int32_t *__restrict__ cnt)
{
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nnzslots) return;
    int32_t c = pat[e];
    if (c >= 0) atomicAdd(cnt + c, 1);
}

__global__ void scan_kernel(const int32_t *__restrict__ cnt, int64_t nr, int32_t *__restrict__ ptr)
{
    __shared__ int64_t part[1024];
    const int t = threadIdx.x;
    const int64_t per = (nr + 1023) / 1024;
    const int64_t a = min(nr, t * per), b = min(nr, a + per);
    int64_t c = 0;
    for (int64_t j = a; j < b; ++j) c += cnt[j];
    part[t] = c;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
        int64_t v = (t >= o) ? part[t - o] : 0;
        __syncthreads();
        part[t] += v;
        __syncthreads();
    }
    int64_t pos = part[t] - c;
    for (int64_t j = a; j < b; ++j) {
        ptr[j] = (int32_t)pos;
        pos += cnt[j];
    }
    if (t == 1023) ptr[nr] = (int32_t)part[1023];
}

__global__ void gt_fill_kernel(const int32_t *__restrict__ pat, int64_t nr, int w,
                               const int32_t *__restrict__ ptr, int32_t *__restrict__ cur,
                               int32_t *__restrict__ row, int32_t *__restrict__ slot)
{
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nr * w) return;
    int32_t c = pat[e];
    if (c < 0) return;
    int32_t pos = ptr[c] + atomicAdd(cur + c, 1);
    row[pos] = (int32_t)(e / w);
    slot[pos] = (int32_t)e;
}

// order each column's entries by row (deterministic G^T products)
__global__ void gt_sort_kernel(const int32_t *__restrict__ ptr, int64_t nr, int32_t *row,
                               int32_t *slot)
{
    int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nr) return;
    int32_t a = ptr[c], b = ptr[c + 1];
    for (int32_t x = a + 1; x < b; ++x) {
        int32_t rv = row[x], sv = slot[x];
        int32_t y = x - 1;
        while (y >= a && row[y] > rv) {
            row[y + 1] = row[y];
            slot[y + 1] = slot[y];
            --y;
        }
        row[y + 1] = rv;
        slot[y + 1] = sv;
    }
}

afn_status transpose_pattern(const int32_t *pat, int64_t nr, int w, int32_t *ptr, int32_t *row,
                             int32_t *slot, cudaStream_t s)
{
    if (nr <= 0) return AFN_OK;
    DevBuf cnt, cur;
    AFN_TRY(cnt.alloc(sizeof(int32_t) * (size_t)nr));
    AFN_TRY(cur.alloc(sizeof(int32_t) * (size_t)nr));
    AFN_CUDA(cudaMemsetAsync(cnt.p, 0, sizeof(int32_t) * nr, s));
    AFN_CUDA(cudaMemsetAsync(cur.p, 0, sizeof(int32_t) * nr, s));
    int64_t slots = nr * w;
    unsigned g = (unsigned)((slots + 255) / 256);
    gt_count_kernel<<<g, 256, 0, s>>>(pat, slots, cnt.as<int32_t>());
    scan_kernel<<<1, 1024, 0, s>>>(cnt.as<int32_t>(), nr, ptr);
    gt_fill_kernel<<<g, 256, 0, s>>>(pat, nr, w, ptr, cur.as<int32_t>(), row, slot);
    gt_sort_kernel<<<(unsigned)((nr + 255) / 256), 256, 0, s>>>(ptr, nr, row, slot);
    AFN_CUDA(cudaGetLastError());
    AFN_CUDA(cudaStreamSynchronize(s));
    return AFN_OK;
}

}  // namespace afn
