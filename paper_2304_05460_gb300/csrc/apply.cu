// apply.cu -- the AFN preconditioner apply s = M^{-1} r (Alg. 3), written in
// terms of W = L^{-1} K12 and the explicit triangular inverses L^{-1}, L^{-T}
// (both formed once at build time):
//   z' = L^{-1} r1
//   t  = r2 - W^T z'          (= r2 - K12^T (K11+mu I)^{-1} r1)
//   s2 = G^T (G t)
//   s1 = L^{-T} (z' - W s2)   (= (K11+mu I)^{-1} (r1 - K12 s2))
// Every product is a streamed pass over one stored operand, so the apply is
// bound by HBM bandwidth: W^T (nr x k) is read twice, L^{-1} and L^{-T} once,
// G twice.  Vectors are n x nrhs column-major (ld = n) in permuted order.
// The two W products of mixed handles run, for a multiple of 16 columns, on
// the tensor cores: on a BF16 image of W with the vectors split into three
// BF16 terms (gemm_bf16.cuh, apply_tc = 2, the default) or three-pass tf32 on
// the FP32 W (gemm_umma.cuh, apply_tc = 1); otherwise, and with apply_tc = 0,
// on the CUDA cores (the gemm_kernel tiles of gemm_tile.cuh; pieces of at
// most 4 columns by rowmul_kernel / colmul_kernel below).
#include <algorithm>
#include <cstring>
#include <type_traits>

#include "afn_device.cuh"
#include "afn_internal.cuh"
#include "gemm_bf16.cuh"
#include "gemm_tile.cuh"
#include "gemm_umma.cuh"
#include "group.cuh"

namespace afn {

// --------------------------------------------------------------------------
// Row-major A times column-major X:  out[i,c] = beta*y[i,c] + alpha*sum_p A[i,p] x[p,c]
// p ranges over [0,K) (TRI=0), [0,i] (TRI=1, lower) or [i,K) (TRI=2, upper).
// One warp per row; lanes stride over p (coalesced rows of A); x is staged
// in shared memory as float4/double2-friendly [c][p] tiles.
// --------------------------------------------------------------------------
static constexpr int RW = 8;       // warps (rows) per CTA
static constexpr int PT = 256;     // p tile

template <class T, int NC, int TRI>
__global__ void __launch_bounds__(RW * 32) rowmul_kernel(const T *__restrict__ A, int64_t lda,
                                                         int64_t M, int64_t K,
                                                         const T *__restrict__ X, int64_t ldx,
                                                         const T *__restrict__ Y, int64_t ldy,
                                                         T *__restrict__ O, int64_t ldo, T alpha,
                                                         T beta)
{
    __shared__ T xs[NC * PT];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t rbase = (int64_t)blockIdx.x * RW;
    const int64_t i = rbase + wid;
    // p range common to the CTA's rows
    int64_t plo = 0, phi = K;
    if (TRI == 1) phi = min(K, rbase + RW);
    if (TRI == 2) plo = rbase;
    T acc[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) acc[c] = 0;
    for (int64_t p0 = plo; p0 < phi; p0 += PT) {
        __syncthreads();
        for (int e = threadIdx.x; e < NC * PT; e += RW * 32) {
            int c = e / PT, pp = e % PT;
            int64_t p = p0 + pp;
            xs[e] = (p < phi) ? X[c * ldx + p] : (T)0;
        }
        __syncthreads();
        if (i < M) {
            for (int pp = lane; pp < PT; pp += 32) {
                int64_t p = p0 + pp;
                if (p >= phi) break;
                if (TRI == 1 && p > i) break;
                if (TRI == 2 && p < i) continue;
                T a = A[i * lda + p];
#pragma unroll
                for (int c = 0; c < NC; ++c) acc[c] += a * xs[c * PT + pp];
            }
        }
    }
    if (i >= M) return;
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        T v = warp_sum(acc[c]);
        if (lane == 0) {
            T base = (beta != (T)0) ? beta * Y[c * ldy + i] : (T)0;
            O[c * ldo + i] = base + alpha * v;
        }
    }
}

// --------------------------------------------------------------------------
// Transposed product with split K:  part[js][c][i] = sum_{j in chunk js} A[j,i] x[j,c]
// (A row-major nrows x ncols; thread per column i: coalesced along rows of A).
// --------------------------------------------------------------------------
static constexpr int CT = 256;     // columns per CTA
static constexpr int JT = 64;      // j tile staged in shared memory

template <class T, int NC>
__global__ void __launch_bounds__(CT) colmul_kernel(const T *__restrict__ A, int64_t lda,
                                                    int64_t nrows, int64_t ncols,
                                                    const T *__restrict__ X, int64_t ldx,
                                                    T *__restrict__ part, int64_t chunk)
{
    __shared__ T xs[JT * NC];
    const int64_t i = (int64_t)blockIdx.x * CT + threadIdx.x;
    const int64_t j0 = (int64_t)blockIdx.y * chunk;
    const int64_t j1 = min(nrows, j0 + chunk);
    T acc[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) acc[c] = 0;
    for (int64_t jt = j0; jt < j1; jt += JT) {
        __syncthreads();
        for (int e = threadIdx.x; e < JT * NC; e += CT) {
            int jj = e / NC, c = e % NC;
            int64_t j = jt + jj;
            xs[e] = (j < j1) ? X[c * ldx + j] : (T)0;
        }
        __syncthreads();
        if (i < ncols) {
            const int jn = (int)min((int64_t)JT, j1 - jt);
            for (int jj = 0; jj < jn; ++jj) {
                T a = A[(jt + jj) * lda + i];
#pragma unroll
                for (int c = 0; c < NC; ++c) acc[c] += a * xs[jj * NC + c];
            }
        }
    }
    if (i >= ncols) return;
#pragma unroll
    for (int c = 0; c < NC; ++c) part[((int64_t)blockIdx.y * NC + c) * ncols + i] = acc[c];
}

// out[i,c] = beta y[i,c] + alpha sum_js part[js][c][i]  (y not read when beta == 0)
template <class T>
__global__ void colmul_finish(const T *__restrict__ part, int js, int nc, int64_t ncols,
                              const T *__restrict__ Y, int64_t ldy, T *__restrict__ O,
                              int64_t ldo, T alpha, T beta)
{
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= ncols * nc) return;
    int c = (int)(e / ncols);
    int64_t i = e % ncols;
    T s = 0;
    for (int q = 0; q < js; ++q) s += part[((int64_t)q * nc + c) * ncols + i];
    const T base = (beta != (T)0) ? beta * Y[c * ldy + i] : (T)0;
    O[c * ldo + i] = base + alpha * s;
}

// ELL product y = G t  (row i: sum_p G[i,p] t[pat[i,p]])
template <class T>
__global__ void spmv_ell_kernel(const T *__restrict__ G, const int32_t *__restrict__ pat,
                                int64_t nr, int w, int nrhs, const T *__restrict__ t, int64_t ldt,
                                T *__restrict__ y, int64_t ldy)
{
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nr * nrhs) return;
    int c = (int)(e / nr);
    int64_t i = e % nr;
    const T *tc = t + c * ldt;
    T s = 0;
    for (int p = 0; p < w; ++p) {
        int32_t j = pat[i * w + p];
        if (j < 0) break;
        s += G[i * w + p] * tc[j];
    }
    y[c * ldy + i] = s;
}

// transposed ELL product s = G^T y through the column lists (ascending row)
template <class T>
__global__ void spmv_gt_kernel(const T *__restrict__ G, const int32_t *__restrict__ ptr,
                               const int32_t *__restrict__ row, const int32_t *__restrict__ slot,
                               int64_t nr, int nrhs, const T *__restrict__ y, int64_t ldy,
                               T *__restrict__ out, int64_t ldo)
{
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nr * nrhs) return;
    int c = (int)(e / nr);
    int64_t j = e % nr;
    const T *yc = y + c * ldy;
    T s = 0;
    for (int32_t q = ptr[j]; q < ptr[j + 1]; ++q) s += G[slot[q]] * yc[row[q]];
    out[c * ldo + j] = s;
}

// Row-major forms of the two sparse products for many right-hand sides: one
// warp per row, lanes over columns.  The row's (index, value) entries are
// loaded 32 at a time by the warp in one coalesced read and handed out by
// shuffles; each entry is then one coalesced gather of the row of t (or y)
// it names, four gathers in flight per lane.  Each output is the sum over the
// row's entries in slot order, the same as a sequential loop.
template <class T, int CB>
__device__ __forceinline__ void sparse_row_rm(const int32_t *__restrict__ idx, const T *__restrict__ val,
                                              int m, int nrhs, const T *__restrict__ src,
                                              T *__restrict__ dst)
{
    const int lane = threadIdx.x & 31;
    for (int cb = 0; cb < nrhs; cb += CB) {
        const int c = cb + lane;
        const bool on = c < nrhs;
        T s = 0;
        for (int p0 = 0; p0 < m; p0 += 32) {
            const int cnt = min(32, m - p0);
            const int32_t jl = lane < cnt ? idx[p0 + lane] : 0;
            const T gl = lane < cnt ? val[p0 + lane] : (T)0;
            int p = 0;
            for (; p + 4 <= cnt; p += 4) {
                const int32_t j0 = __shfl_sync(0xffffffffu, jl, p), j1 = __shfl_sync(0xffffffffu, jl, p + 1);
                const int32_t j2 = __shfl_sync(0xffffffffu, jl, p + 2), j3 = __shfl_sync(0xffffffffu, jl, p + 3);
                const T g0 = __shfl_sync(0xffffffffu, gl, p), g1 = __shfl_sync(0xffffffffu, gl, p + 1);
                const T g2 = __shfl_sync(0xffffffffu, gl, p + 2), g3 = __shfl_sync(0xffffffffu, gl, p + 3);
                T v0 = 0, v1 = 0, v2 = 0, v3 = 0;
                if (on) {
                    v0 = src[(int64_t)j0 * nrhs + c];
                    v1 = src[(int64_t)j1 * nrhs + c];
                    v2 = src[(int64_t)j2 * nrhs + c];
                    v3 = src[(int64_t)j3 * nrhs + c];
                }
                s += g0 * v0;
                s += g1 * v1;
                s += g2 * v2;
                s += g3 * v3;
            }
            for (; p < cnt; ++p) {
                const int32_t j = __shfl_sync(0xffffffffu, jl, p);
                const T g = __shfl_sync(0xffffffffu, gl, p);
                if (on) s += g * src[(int64_t)j * nrhs + c];
            }
        }
        if (on) dst[c] = s;
    }
}

template <class T>
__global__ void spmv_ell_rm_kernel(const T *__restrict__ G, const int32_t *__restrict__ pat,
                                   int64_t nr, int w, int nrhs, const T *__restrict__ trm,
                                   T *__restrict__ yrm)
{
    const int64_t i = (int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    if (i >= nr) return;
    // used slots: i + 1 for the short first rows, w after them (diagonal last)
    const int m = (int)min((int64_t)w, i + 1);
    sparse_row_rm<T, 32>(pat + i * w, G + i * w, m, nrhs, trm, yrm + i * nrhs);
}

// s = G^T y through the column lists of G (ascending row), with the values
// copied into list order (gtv) so that each entry is read where it is listed
template <class T>
__global__ void spmv_gt_rm_kernel(const T *__restrict__ gtv, const int32_t *__restrict__ ptr,
                                  const int32_t *__restrict__ row, int64_t nr, int nrhs,
                                  const T *__restrict__ yrm, T *__restrict__ orm)
{
    const int64_t j = (int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    if (j >= nr) return;
    const int32_t q0 = ptr[j], q1 = ptr[j + 1];
    sparse_row_rm<T, 32>(row + q0, gtv + q0, q1 - q0, nrhs, yrm, orm + j * nrhs);
}

// gtv[q] = G[slot[q]]: the values of G in the order of the column lists
template <class T>
__global__ void gt_values_kernel(const T *__restrict__ G, const int32_t *__restrict__ slot,
                                 int64_t nnz, T *__restrict__ gtv)
{
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q < nnz) gtv[q] = G[slot[q]];
}

afn_status make_gt_values(Handle *h, cudaStream_t s)
{
    const int64_t nr = h->nr;
    if (nr <= 0 || !h->gt_ptr.p) return AFN_OK;
    int32_t nnz = 0;
    AFN_CUDA(cudaMemcpyAsync(&nnz, h->gt_ptr.as<int32_t>() + nr, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    AFN_CUDA(cudaStreamSynchronize(s));
    const unsigned g = (unsigned)((nnz + 255) / 256);
    if (h->G.p && h->precision != AFN_PREC_MIXED) {     // the FP64 apply
        AFN_TRY(h->gtv.alloc(sizeof(double) * (size_t)std::max(nnz, 1)));
        if (nnz) gt_values_kernel<double><<<g, 256, 0, s>>>(h->G.as<double>(), h->gt_slot.as<int32_t>(), nnz,
                                                            h->gtv.as<double>());
    }
    if (h->G32.p) {
        AFN_TRY(h->gtv32.alloc(sizeof(float) * (size_t)std::max(nnz, 1)));
        if (nnz) gt_values_kernel<float><<<g, 256, 0, s>>>(h->G32.as<float>(), h->gt_slot.as<int32_t>(), nnz,
                                                           h->gtv32.as<float>());
    }
    AFN_CUDA(cudaGetLastError());
    return AFN_OK;
}

// out[i*cols + c] = in[c*ldin + i]  (column-major -> row-major), 32x32 tiles
template <class T>
__global__ void cm_to_rm_kernel(const T *__restrict__ in, int64_t ldin, int64_t rows, int cols,
                                T *__restrict__ out)
{
    __shared__ T t[32][33];
    const int64_t i0 = (int64_t)blockIdx.x * 32;
    const int c0 = blockIdx.y * 32;
    for (int q = threadIdx.y; q < 32; q += blockDim.y) {
        int c = c0 + q;
        int64_t i = i0 + threadIdx.x;
        if (c < cols && i < rows) t[q][threadIdx.x] = in[c * ldin + i];
    }
    __syncthreads();
    for (int q = threadIdx.y; q < 32; q += blockDim.y) {
        int64_t i = i0 + q;
        int c = c0 + threadIdx.x;
        if (c < cols && i < rows) out[i * cols + c] = t[threadIdx.x][q];
    }
}

// out[c*ldout + i] = in[i*cols + c]  (row-major -> column-major)
template <class T>
__global__ void rm_to_cm_kernel(const T *__restrict__ in, int64_t rows, int cols,
                                T *__restrict__ out, int64_t ldout)
{
    __shared__ T t[32][33];
    const int64_t i0 = (int64_t)blockIdx.x * 32;
    const int c0 = blockIdx.y * 32;
    for (int q = threadIdx.y; q < 32; q += blockDim.y) {
        int64_t i = i0 + q;
        int c = c0 + threadIdx.x;
        if (c < cols && i < rows) t[q][threadIdx.x] = in[i * cols + c];
    }
    __syncthreads();
    for (int q = threadIdx.y; q < 32; q += blockDim.y) {
        int c = c0 + q;
        int64_t i = i0 + threadIdx.x;
        if (c < cols && i < rows) out[c * ldout + i] = t[threadIdx.x][q];
    }
}

// --------------------------------------------------------------------------
// Tiled product for many right-hand sides (NC in {8, 16, 32}), see gemm_rows:
// a CTA owns GM = 128 output rows and one K-chunk.  With one K-chunk the
// epilogue writes O = beta Y + alpha acc directly; otherwise per-chunk
// partials go to `part` (chunk-major) and gemm_finish sums them in order.
// --------------------------------------------------------------------------
template <class T, int NC, bool TA, int TRI>
__global__ void __launch_bounds__(256) gemm_kernel(const T *__restrict__ A, int64_t lda, int64_t M,
                                                   int64_t K, const T *__restrict__ X,
                                                   int64_t ldx, int64_t chunk,
                                                   T *__restrict__ part, const T *__restrict__ Y,
                                                   int64_t ldy, T *__restrict__ O, int64_t ldo,
                                                   T alpha, T beta)
{
    constexpr int TC = GemmShape<NC>::TC;
    constexpr int RM = GemmShape<NC>::RM;
    __shared__ __align__(16) T as[GK][GM + 4];
    __shared__ __align__(16) T xs[GK][NC + 4];
    const int tc = threadIdx.x % TC, tr = threadIdx.x / TC;
    const int64_t r0 = (int64_t)blockIdx.x * GM;
    const int64_t k0 = (int64_t)blockIdx.y * chunk;
    const int64_t k1 = min(K, k0 + chunk);
    T acc[RM][4];
    gemm_rows<T, NC, TA, TRI>(A, lda, M, r0, k0, k1, X, ldx, as, xs, acc);
#pragma unroll
    for (int a = 0; a < RM; ++a) {
        int64_t gi = r0 + tr * RM + a;
        if (gi >= M) continue;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            int c = tc * 4 + b;
            if (gridDim.y == 1) {
                T base = (beta != (T)0) ? beta * Y[c * ldy + gi] : (T)0;
                O[c * ldo + gi] = base + alpha * acc[a][b];
            } else {
                part[((int64_t)blockIdx.y * NC + c) * M + gi] = acc[a][b];
            }
        }
    }
}

// O[i,c] = beta Y[i,c] + alpha sum_q part[q][c][i]
template <class T>
__global__ void gemm_finish(const T *__restrict__ part, int js, int nc, int64_t M,
                            const T *__restrict__ Y, int64_t ldy, T *__restrict__ O, int64_t ldo,
                            T alpha, T beta)
{
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= M * nc) return;
    int c = (int)(e / M);
    int64_t i = e % M;
    T s = 0;
    for (int q = 0; q < js; ++q) s += part[((int64_t)q * nc + c) * M + i];
    T base = (beta != (T)0) ? beta * Y[c * ldy + i] : (T)0;
    O[c * ldo + i] = base + alpha * s;
}

template <class T>
__global__ void copy_cols_kernel(const T *__restrict__ a, int64_t lda, T *__restrict__ b,
                                 int64_t ldb, int64_t rows, int nrhs)
{
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= rows * nrhs) return;
    int c = (int)(e / rows);
    int64_t i = e % rows;
    b[c * ldb + i] = a[c * lda + i];
}

static int piece(int left, int cap)
{
    int b = 1;
    while (b * 2 <= left && b * 2 <= cap) b *= 2;
    return b;
}

template <class T, int TRI>
static void rowmul(const T *A, int64_t lda, int64_t M, int64_t K, const T *X, int64_t ldx,
                   const T *Y, int64_t ldy, T *O, int64_t ldo, T alpha, T beta, int nrhs,
                   cudaStream_t s)
{
    unsigned g = (unsigned)((M + RW - 1) / RW);
    for (int c0 = 0; c0 < nrhs;) {
        int b = piece(nrhs - c0, sizeof(T) == 8 ? 8 : 16);
        const T *x = X + c0 * ldx;
        const T *y = Y ? Y + c0 * ldy : nullptr;
        T *o = O + c0 * ldo;
        switch (b) {
        case 1: rowmul_kernel<T, 1, TRI><<<g, RW * 32, 0, s>>>(A, lda, M, K, x, ldx, y, ldy, o, ldo, alpha, beta); break;
        case 2: rowmul_kernel<T, 2, TRI><<<g, RW * 32, 0, s>>>(A, lda, M, K, x, ldx, y, ldy, o, ldo, alpha, beta); break;
        case 4: rowmul_kernel<T, 4, TRI><<<g, RW * 32, 0, s>>>(A, lda, M, K, x, ldx, y, ldy, o, ldo, alpha, beta); break;
        case 8: rowmul_kernel<T, 8, TRI><<<g, RW * 32, 0, s>>>(A, lda, M, K, x, ldx, y, ldy, o, ldo, alpha, beta); break;
        default: rowmul_kernel<T, 16, TRI><<<g, RW * 32, 0, s>>>(A, lda, M, K, x, ldx, y, ldy, o, ldo, alpha, beta); break;
        }
        c0 += b;
    }
}

static int colmul_js(int64_t nrows, int64_t ncols)
{
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int64_t cb = (ncols + CT - 1) / CT;
    int64_t js = (sms * 8 + cb - 1) / cb;
    js = std::min<int64_t>(js, std::max<int64_t>(1, nrows / (4 * JT)));
    return (int)std::max<int64_t>(1, std::min<int64_t>(js, 128));
}

static constexpr int GEMM_JS_MAX = 64;

// words of the split vector block of the tcgen05 products (both products):
// tf32 hi/lo of 32 columns (64 words per K-element) or three BF16 terms of
// 64 columns (96 words per K-element)
static int64_t gu_bk_words(int64_t nr, int64_t k)
{
    return 96 * ((std::max(nr, k) + GKB - 1) / GKB * GKB);
}

// split-K partials of the products, elements: the CUDA-core tiles' chunks of
// the k-row products, or one 64-column partial of the n_r-row product
static size_t apply_pcap(int64_t nr, int64_t k)
{
    const size_t a = (size_t)std::max(colmul_js(nr, k), GEMM_JS_MAX) * 32 * (size_t)std::max<int64_t>(k, 1);
    return std::max(a, (size_t)64 * (size_t)std::max(nr, k));
}

size_t apply_tmp_elems(const Handle *h, int nrhs)
{
    int64_t k = h->k, nr = h->nr;
    // zp, u (k x nrhs), t, y (nr x nrhs), GEMM partials, row-major copy (nr x nrhs), split
    // vector block of the tcgen05 products
    return (size_t)(2 * k * nrhs + 3 * nr * nrhs) + apply_pcap(nr, k) + (size_t)gu_bk_words(nr, k) + 64;
}

// ------------------------------------------------ tcgen05 W products --------
// Atl (see gemm32u_kernel): A[row][kk] = Wt[row k + kk] (trans = 0, M = nr,
// K = k) or Wt[kk k + row] (trans = 1, M = k, K = nr), zero outside
__global__ void gu_arrange_kernel(const float *__restrict__ Wt, int64_t k, int trans, int64_t M,
                                  int64_t K, int64_t nks, float *__restrict__ Atl, int64_t total)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= total) return;
    const int64_t per = nks * (UR * GKU);
    const int64_t rt = e / per, rem = e % per;
    const int64_t st = rem / (UR * GKU);
    const int wd = (int)(rem % (UR * GKU));
    const int row = (wd / ((GKU / 4) * 32)) * 8 + (wd % 32) / 4;
    const int kk = ((wd % ((GKU / 4) * 32)) / 32) * 4 + wd % 4;
    const int64_t gi = rt * UR + row, gk = st * GKU + kk;
    float v = 0.f;
    if (gi < M && gk < K) v = trans ? Wt[gk * k + gi] : Wt[gi * k + gk];
    Atl[e] = v;
}

// Bk: the K x NR block of X (column-major, leading dimension ldx) split into
// tf32 hi / lo, per stage of GKU rows the hi then lo halves in the K-major
// core-matrix layout of gemm32u_kernel, zero past K
template <int NR>
__global__ void gu_bsplit_kernel(const float *__restrict__ X, int64_t ldx, int64_t K, int64_t nks,
                                 uint32_t *__restrict__ Bk)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t kp = nks * GKU;
    if (e >= kp * NR) return;
    const int64_t kg = e % kp;
    const int c = (int)(e / kp);
    uint32_t hi, lo;
    tf32_split(kg < K ? X[c * ldx + kg] : 0.f, hi, lo);
    const int64_t st = kg / GKU;
    const int kk = (int)(kg % GKU);
    const int64_t w = st * (2 * GKU * NR) + (c / 8) * (GKU / 4) * 32 + (kk / 4) * 32 + (c % 8) * 4 +
                      (kk % 4);
    Bk[w] = hi;
    Bk[w + GKU * NR] = lo;
}

// the handle's option apply_tc: 1 runs the W products on the tensor cores in
// three-pass tf32, 2 with BF16 images of W
static int apply_tc_mode(const Handle *h) { return h->opt.apply_tc; }

// BF16 image (see gemm16u_kernel): A[row][kk] = Wt[row k + kk] (trans = 0,
// M = nr, K = k) or Wt[kk k + row] (trans = 1, M = k, K = nr), zero outside
__global__ void gb_arrange_kernel(const float *__restrict__ Wt, int64_t k, int trans, int64_t M,
                                  int64_t K, int64_t nks, __nv_bfloat16 *__restrict__ Atl,
                                  int64_t total)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= total) return;
    const int64_t per = nks * (UR * GKB);
    const int64_t rt = e / per, rem = e % per;
    const int64_t st = rem / (UR * GKB);
    const int wd = (int)(rem % (UR * GKB));
    const int cm = wd / 64, within = wd % 64;
    const int row = (cm / (GKB / 8)) * 8 + within / 8;
    const int kk = (cm % (GKB / 8)) * 8 + within % 8;
    const int64_t gi = rt * UR + row, gk = st * GKB + kk;
    float v = 0.f;
    if (gi < M && gk < K) v = trans ? Wt[gk * k + gi] : Wt[gi * k + gk];
    Atl[e] = __float2bfloat16_rn(v);
}

// Bk: the K x NC block of X (column-major, leading dimension ldx) split into
// NT BF16 terms, term t of column c at column t NC + c of the stage tile,
// zero past K
template <int NC, int NT>
__global__ void gb_bsplit_kernel(const float *__restrict__ X, int64_t ldx, int64_t K, int64_t nks,
                                 __nv_bfloat16 *__restrict__ Bk)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t kp = nks * GKB;
    if (e >= kp * NC) return;
    const int64_t kg = e % kp;
    const int c = (int)(e / kp);
    float x = kg < K ? X[c * ldx + kg] : 0.f;
    const int64_t st = kg / GKB;
    const int kk = (int)(kg % GKB);
    __nv_bfloat16 *stage = Bk + st * (int64_t)(GKB * NC * NT);
#pragma unroll
    for (int t = 0; t < NT; ++t) {
        const __nv_bfloat16 b = __float2bfloat16_rn(x);
        stage[gb_tile_elem(t * NC + c, kk)] = b;
        x -= __bfloat162float(b);
    }
}

static int64_t gu_nks(int64_t K) { return (K + GKU - 1) / GKU; }
static int64_t gu_tiles(int64_t M) { return (M + UR - 1) / UR; }

static int64_t gb_nks(int64_t K) { return (K + GKB - 1) / GKB; }

afn_status apply_tc_prepare(Handle *h, cudaStream_t s)
{
    if (h->wu_tried || apply_tc_mode(h) == 0) return AFN_OK;
    h->wu_tried = true;
    const int64_t k = h->k, nr = h->nr;
    // small products stay on the CUDA-core tiles
    if (!h->Wt32.p || k < 128 || nr < 128) return AFN_OK;
    if (apply_tc_mode(h) == 2) {
        const int64_t n1 = gu_tiles(nr) * gb_nks(k) * (UR * GKB);
        const int64_t n2 = gu_tiles(k) * gb_nks(nr) * (UR * GKB);
        AFN_TRY(h->Wb1.alloc(sizeof(__nv_bfloat16) * (size_t)n1));
        AFN_TRY(h->Wb2.alloc(sizeof(__nv_bfloat16) * (size_t)n2));
        gb_arrange_kernel<<<(unsigned)((n1 + 255) / 256), 256, 0, s>>>(
            h->Wt32.as<float>(), k, 0, nr, k, gb_nks(k), h->Wb1.as<__nv_bfloat16>(), n1);
        gb_arrange_kernel<<<(unsigned)((n2 + 255) / 256), 256, 0, s>>>(
            h->Wt32.as<float>(), k, 1, k, nr, gb_nks(nr), h->Wb2.as<__nv_bfloat16>(), n2);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(e, "apply BF16 images");
        return AFN_OK;
    }
    const int64_t n1 = gu_tiles(nr) * gu_nks(k) * (UR * GKU);
    const int64_t n2 = gu_tiles(k) * gu_nks(nr) * (UR * GKU);
    AFN_TRY(h->Wu1.alloc(sizeof(float) * (size_t)n1));
    AFN_TRY(h->Wu2.alloc(sizeof(float) * (size_t)n2));
    gu_arrange_kernel<<<(unsigned)((n1 + 255) / 256), 256, 0, s>>>(h->Wt32.as<float>(), k, 0, nr, k,
                                                                   gu_nks(k), h->Wu1.as<float>(), n1);
    gu_arrange_kernel<<<(unsigned)((n2 + 255) / 256), 256, 0, s>>>(h->Wt32.as<float>(), k, 1, k, nr,
                                                                   gu_nks(nr), h->Wu2.as<float>(), n2);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "apply tile images");
    return AFN_OK;
}

// j-chunks of a tcgen05 product: 1 CTA per SM; the count whose CTAs fill the
// last wave best, chunks of at least 8 stages, partials within cap
static void gu_chunking(int64_t M, int64_t nks, size_t cap_words, int nr, int &js, int64_t &cs,
                        int per_sm = 1)
{
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    sms *= per_sm;
    const int64_t rt = gu_tiles(M);
    double best = -1.0;
    js = 1;
    cs = nks;
    for (int q = 1; q <= 64; ++q) {
        const int64_t c = (nks + q - 1) / q;
        if (q > 1 && c < 8) break;
        const int64_t jq = (nks + c - 1) / c;
        if ((size_t)jq * (size_t)nr * (size_t)M > cap_words) break;
        const int64_t tot = rt * jq, waves = (tot + sms - 1) / sms;
        const double eff = (double)tot / (double)(waves * sms);
        if (eff > best + 1e-9) {
            best = eff;
            js = (int)jq;
            cs = c;
        }
    }
}

// O = beta Y + alpha A X on the tensor cores for nrhs columns (a multiple of 16)
static afn_status prod_tc(const float *Atl, int64_t M, int64_t K, const float *X, int64_t ldx,
                          const float *Y, int64_t ldy, float *O, int64_t ldo, float alpha, float beta,
                          int nrhs, float *part, size_t pcap, uint32_t *Bk, int *err, cudaStream_t s)
{
    const int64_t nks = gu_nks(K);
    for (int c0 = 0; c0 < nrhs;) {
        const int b = (nrhs - c0) >= 32 ? 32 : 16;
        int js;
        int64_t cs;
        gu_chunking(M, nks, pcap, b, js, cs);
        const int64_t tot = nks * GKU * b;
        dim3 grid((unsigned)gu_tiles(M), (unsigned)js);
        if (b == 32) {
            gu_bsplit_kernel<32><<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(X + c0 * ldx, ldx, K, nks, Bk);
            const int smem = GNST * GStage<32>::BYTES;
            cudaFuncSetAttribute(gemm32u_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
            gemm32u_kernel<4><<<grid, GUT, smem, s>>>(Atl, M, nks, Bk, part, cs, err, wait_limit_ns());
        } else {
            gu_bsplit_kernel<16><<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(X + c0 * ldx, ldx, K, nks, Bk);
            const int smem = GNST * GStage<16>::BYTES;
            cudaFuncSetAttribute(gemm32u_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
            gemm32u_kernel<2><<<grid, GUT, smem, s>>>(Atl, M, nks, Bk, part, cs, err, wait_limit_ns());
        }
        const int64_t te = M * b;
        gemm_finish<float><<<(unsigned)((te + 255) / 256), 256, 0, s>>>(
            part, js, b, M, Y ? Y + c0 * ldy : nullptr, ldy, O + c0 * ldo, ldo, alpha, beta);
        c0 += b;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "tcgen05 apply product");
    return AFN_OK;
}

// O = beta Y + alpha A X on the BF16 tensor cores for nrhs columns (a multiple of 16)
template <int NC>
static void launch_g16(const __nv_bfloat16 *Atl, int64_t M, int64_t nks, const float *X, int64_t ldx,
                       int64_t K, float *part, size_t pcap, __nv_bfloat16 *Bk, int *err, int &js,
                       cudaStream_t s)
{
    constexpr int NT = 3;
    constexpr int smem = GBNST * GbStage<NC, NT>::BYTES;
    int64_t cs;
    gu_chunking(M, nks, pcap, NC, js, cs, smem <= 112 * 1024 ? 2 : 1);
    const int64_t tot = nks * GKB * NC;
    gb_bsplit_kernel<NC, NT><<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(X, ldx, K, nks, Bk);
    cudaFuncSetAttribute(gemm16u_kernel<NC, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    dim3 grid((unsigned)gu_tiles(M), (unsigned)js);
    gemm16u_kernel<NC, NT><<<grid, GBT, smem, s>>>(Atl, M, nks, Bk, part, cs, err, wait_limit_ns());
}

static afn_status prod_bf16(const __nv_bfloat16 *Atl, int64_t M, int64_t K, const float *X, int64_t ldx,
                            const float *Y, int64_t ldy, float *O, int64_t ldo, float alpha, float beta,
                            int nrhs, float *part, size_t pcap, __nv_bfloat16 *Bk, int *err,
                            cudaStream_t s)
{
    const int64_t nks = gb_nks(K);
    for (int c0 = 0; c0 < nrhs;) {
        const int left = nrhs - c0;
        const int b = left >= 64 ? 64 : (left >= 32 ? 32 : 16);
        int js = 1;
        const float *x = X + (int64_t)c0 * ldx;
        if (b == 64) launch_g16<64>(Atl, M, nks, x, ldx, K, part, pcap, Bk, err, js, s);
        else if (b == 32) launch_g16<32>(Atl, M, nks, x, ldx, K, part, pcap, Bk, err, js, s);
        else launch_g16<16>(Atl, M, nks, x, ldx, K, part, pcap, Bk, err, js, s);
        const int64_t te = M * b;
        gemm_finish<float><<<(unsigned)((te + 255) / 256), 256, 0, s>>>(
            part, js, b, M, Y ? Y + (int64_t)c0 * ldy : nullptr, ldy, O + (int64_t)c0 * ldo, ldo, alpha,
            beta);
        c0 += b;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "BF16 tensor-core apply product");
    return AFN_OK;
}

static int gemm_js(int64_t M, int64_t K)
{
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int64_t mb = (M + GM - 1) / GM;
    int64_t js = (4 * (int64_t)sms + mb - 1) / mb;
    js = std::min<int64_t>(js, std::max<int64_t>(1, K / 256));
    return (int)std::max<int64_t>(1, std::min<int64_t>(js, GEMM_JS_MAX));
}

// out = beta Y + alpha op(A) X for nrhs columns (op(A) = A or A^T, TRI as in
// gemm_kernel); part holds GEMM_JS_MAX * 32 * M elements of scratch.
template <class T, bool TA, int TRI>
static void prod(const T *A, int64_t lda, int64_t M, int64_t K, const T *X, int64_t ldx,
                 const T *Y, int64_t ldy, T *O, int64_t ldo, T alpha, T beta, int nrhs, T *part,
                 size_t part_cap, cudaStream_t s)
{
    for (int c0 = 0; c0 < nrhs;) {
        int left = nrhs - c0;
        const T *x = X + c0 * ldx;
        const T *y = Y ? Y + c0 * ldy : nullptr;
        T *o = O + c0 * ldo;
        if (left >= 8) {
            int b = left >= 32 ? 32 : (left >= 16 ? 16 : 8);
            int js = gemm_js(M, K);
            js = (int)std::max<int64_t>(1, std::min<int64_t>(js, (int64_t)(part_cap / ((size_t)b * M))));
            int64_t chunk = (K + js - 1) / js;
            chunk = (chunk + GK - 1) / GK * GK;
            js = (int)std::max<int64_t>(1, (K + chunk - 1) / chunk);
            dim3 grid((unsigned)((M + GM - 1) / GM), (unsigned)js);
#define GL(NC) gemm_kernel<T, NC, TA, TRI><<<grid, 256, 0, s>>>(A, lda, M, K, x, ldx, chunk, part, \
                                                                 y, ldy, o, ldo, alpha, beta)
            if (b == 32) GL(32); else if (b == 16) GL(16); else GL(8);
#undef GL
            if (js > 1) {
                int64_t tot = M * b;
                gemm_finish<T><<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(part, js, b, M, y, ldy,
                                                                            o, ldo, alpha, beta);
            }
            c0 += b;
            continue;
        }
        int b = piece(left, 4);
        if (!TA) {
            rowmul<T, TRI>(A, lda, M, K, x, ldx, y, ldy, o, ldo, alpha, beta, b, s);
        } else {
            // transposed tail: split-K column kernel, then o = beta y + alpha sum
            int js = colmul_js(K, M);
            js = (int)std::max<int64_t>(1, std::min<int64_t>(js, (int64_t)(part_cap / ((size_t)b * M))));
            int64_t chunk = (K + js - 1) / js;
            js = (int)((K + chunk - 1) / chunk);
            dim3 grid((unsigned)((M + CT - 1) / CT), (unsigned)js);
            switch (b) {
            case 1: colmul_kernel<T, 1><<<grid, CT, 0, s>>>(A, lda, K, M, x, ldx, part, chunk); break;
            case 2: colmul_kernel<T, 2><<<grid, CT, 0, s>>>(A, lda, K, M, x, ldx, part, chunk); break;
            default: colmul_kernel<T, 4><<<grid, CT, 0, s>>>(A, lda, K, M, x, ldx, part, chunk); break;
            }
            int64_t tot = M * b;
            colmul_finish<T><<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(part, js, b, M, y, ldy, o,
                                                                           ldo, alpha, beta);
        }
        c0 += b;
    }
}

// ------------------------------------------------------- Nystrom branch ----
template <class T>
__global__ void scale_cols_kernel(const T *__restrict__ a, int64_t n, int nrhs, int64_t ld, T f,
                                  T *__restrict__ out)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n * nrhs) return;
    const int64_t c = e / n, i = e % n;
    out[c * ld + i] = a[c * ld + i] * f;
}

__global__ void add_diag_kernel(double *C, int64_t k, double v)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < k) C[i * k + i] += v;
}

afn_status nystrom_factor(Handle *h, cudaStream_t s)
{
    const int64_t n = h->n, k = h->k;
    if (k == 0) return AFN_OK;
    // C = B^T B from the row-major B and a column-major copy, then mu on the diagonal
    DevBuf bcm, part;
    AFN_TRY(bcm.alloc(sizeof(double) * (size_t)(n * k)));
    dim3 tb(32, 8), tg((unsigned)((n + 31) / 32), (unsigned)((k + 31) / 32));
    rm_to_cm_kernel<double><<<tg, tb, 0, s>>>(h->Bn.as<double>(), n, (int)k, bcm.as<double>(), n);
    const size_t pcap = (size_t)GEMM_JS_MAX * 32 * (size_t)k;
    AFN_TRY(part.alloc(sizeof(double) * pcap));
    DevBuf Cm;
    AFN_TRY(Cm.alloc(sizeof(double) * (size_t)(k * k)));
    prod<double, true, 0>(h->Bn.as<double>(), k, k, n, bcm.as<double>(), n, nullptr, 0,
                          Cm.as<double>(), k, 1.0, 0.0, (int)k, part.as<double>(), pcap, s);
    add_diag_kernel<<<(unsigned)((k + 255) / 256), 256, 0, s>>>(Cm.as<double>(), k, h->mu);
    AFN_TRY(cholesky64(Cm.as<double>(), k, h->status.as<int>(), s, -1.0));
    AFN_TRY(sync_status(h, "Cholesky of mu I + B^T B"));
    AFN_TRY(h->LcInv.alloc(sizeof(double) * (size_t)(k * k)));
    AFN_TRY(h->LcInvT.alloc(sizeof(double) * (size_t)(k * k)));
    AFN_TRY(tri_inverse64(Cm.as<double>(), k, h->LcInv.as<double>(), h->LcInvT.as<double>(), s));
    if (h->precision == AFN_PREC_MIXED) {
        AFN_TRY(h->Bn32.alloc(sizeof(float) * (size_t)(n * k)));
        AFN_TRY(h->LcInv32.alloc(sizeof(float) * (size_t)(k * k)));
        AFN_TRY(h->LcInvT32.alloc(sizeof(float) * (size_t)(k * k)));
        AFN_TRY(convert64to32(h->Bn.as<double>(), h->Bn32.as<float>(), n * k, s));
        AFN_TRY(convert64to32(h->LcInv.as<double>(), h->LcInv32.as<float>(), k * k, s));
        AFN_TRY(convert64to32(h->LcInvT.as<double>(), h->LcInvT32.as<float>(), k * k, s));
    }
    AFN_CUDA(cudaStreamSynchronize(s));   // the temporaries go out of scope
    return AFN_OK;
}

// s = (K_nys + mu I)^{-1} r = (r - B Lc^{-T} Lc^{-1} B^T r) / mu  (eq. (nystrom1-smw) through
// the SMW identity), vectors in the permuted order
template <class T>
static afn_status nystrom_apply(const Handle *h, const T *r, int nrhs, T *s, T *tmp, cudaStream_t st)
{
    const int64_t n = h->n, k = h->k, nr = h->nr;
    const T f = (T)(1.0 / h->mu);
    if (k > 0) {
        const bool dbl = std::is_same<T, double>::value;
        const T *B = reinterpret_cast<const T *>(dbl ? h->Bn.p : h->Bn32.p);
        const T *Li = reinterpret_cast<const T *>(dbl ? h->LcInv.p : h->LcInv32.p);
        const T *LiT = reinterpret_cast<const T *>(dbl ? h->LcInvT.p : h->LcInvT32.p);
        if (!B || !Li || !LiT) {
            set_error("nystrom apply: factors missing for this precision");
            return AFN_ERR_ARG;
        }
        T *y = tmp, *v = tmp + k * nrhs;
        T *part = tmp + 2 * k * nrhs + 2 * nr * nrhs;
        const size_t pcap = apply_pcap(nr, k);
        prod<T, true, 0>(B, k, k, n, r, n, nullptr, 0, y, k, (T)1, (T)0, nrhs, part, pcap, st);
        prod<T, false, 1>(Li, k, k, k, y, k, nullptr, 0, v, k, (T)1, (T)0, nrhs, part, pcap, st);
        prod<T, false, 2>(LiT, k, k, k, v, k, nullptr, 0, y, k, (T)1, (T)0, nrhs, part, pcap, st);
        prod<T, false, 0>(B, k, n, k, y, k, r, n, s, n, (T)-1, (T)1, nrhs, part, pcap, st);
        const int64_t tot = n * nrhs;
        scale_cols_kernel<T><<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(s, n, nrhs, n, f, s);
    } else {
        const int64_t tot = n * nrhs;
        scale_cols_kernel<T><<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(r, n, nrhs, n, f, s);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "nystrom apply launch");
    return AFN_OK;
}

template <class T>
afn_status afn_apply(const Handle *h, const T *Linv, const T *LinvT, const T *Wt, const T *G,
                     const T *r, int nrhs, T *s, T *tmp, cudaStream_t st)
{
    if (h->precond == AFN_PRECOND_NYSTROM) return nystrom_apply<T>(h, r, nrhs, s, tmp, st);
    const int64_t n = h->n, k = h->k, nr = h->nr;
    const int w = h->w;
    T *zp = tmp;                       // k x nrhs
    T *u = zp + k * nrhs;              // k x nrhs
    T *t = u + k * nrhs;               // nr x nrhs
    T *y = t + nr * nrhs;              // nr x nrhs
    T *part = y + nr * nrhs;           // GEMM_JS_MAX x 32 x k
    const size_t pcap = apply_pcap(nr, k);
    const T *r1 = r, *r2 = r + k;
    T *s1 = s, *s2 = s + k;
    // tcgen05 W products (mixed handles with tiled images, 16-column pieces):
    // mode 1 three-pass tf32 on the FP32 images, mode 2 the BF16 images
    int tc = 0;
    if (std::is_same<T, float>::value && nrhs % 16 == 0) {
        if (apply_tc_mode(h) == 1 && h->Wu1.p && h->Wu2.p) tc = 1;
        if (apply_tc_mode(h) == 2 && h->Wb1.p && h->Wb2.p) tc = 2;
    }
    uint32_t *Bk = reinterpret_cast<uint32_t *>(part + pcap + nr * nrhs);
    __nv_bfloat16 *Bk16 = reinterpret_cast<__nv_bfloat16 *>(Bk);
    int *err = h->status.as<int>() + 3;
    if (k > 0) prod<T, false, 1>(Linv, k, k, k, r1, n, nullptr, 0, zp, k, (T)1, (T)0, nrhs, part, pcap, st);
    if (nr > 0) {
        if (k > 0 && tc == 1) {
            if constexpr (std::is_same<T, float>::value)
                AFN_TRY(prod_tc(h->Wu1.as<float>(), nr, k, zp, k, r2, n, t, nr, -1.f, 1.f, nrhs, part,
                                pcap, Bk, err, st));
        } else if (k > 0 && tc == 2) {
            if constexpr (std::is_same<T, float>::value)
                AFN_TRY(prod_bf16(h->Wb1.as<__nv_bfloat16>(), nr, k, zp, k, r2, n, t, nr, -1.f, 1.f,
                                  nrhs, part, pcap, Bk16, err, st));
        } else if (k > 0) prod<T, false, 0>(Wt, k, nr, k, zp, k, r2, n, t, nr, (T)-1, (T)1, nrhs, part, pcap, st);
        else {
            int64_t tot = nr * nrhs;
            copy_cols_kernel<T><<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(r2, n, t, nr, nr, nrhs);
        }
        int64_t tot = nr * nrhs;
        if (nrhs >= 8) {
            // row-major copies: t -> trm, G trm -> y (row-major), G^T y -> trm -> s2
            T *trm = part + pcap;
            dim3 tb(32, 8), tg((unsigned)((nr + 31) / 32), (unsigned)((nrhs + 31) / 32));
            unsigned gw = (unsigned)((nr + 7) / 8);
            cm_to_rm_kernel<T><<<tg, tb, 0, st>>>(t, nr, nr, nrhs, trm);
            spmv_ell_rm_kernel<T><<<gw, 256, 0, st>>>(G, h->pat.as<int32_t>(), nr, w, nrhs, trm, y);
            const T *gtv = reinterpret_cast<const T *>(std::is_same<T, float>::value ? h->gtv32.p : h->gtv.p);
            spmv_gt_rm_kernel<T><<<gw, 256, 0, st>>>(gtv, h->gt_ptr.as<int32_t>(), h->gt_row.as<int32_t>(),
                                                     nr, nrhs, y, trm);
            rm_to_cm_kernel<T><<<tg, tb, 0, st>>>(trm, nr, nrhs, s2, n);
        } else {
            unsigned g = (unsigned)((tot + 255) / 256);
            spmv_ell_kernel<T><<<g, 256, 0, st>>>(G, h->pat.as<int32_t>(), nr, w, nrhs, t, nr, y, nr);
            spmv_gt_kernel<T><<<g, 256, 0, st>>>(G, h->gt_ptr.as<int32_t>(), h->gt_row.as<int32_t>(),
                                                 h->gt_slot.as<int32_t>(), nr, nrhs, y, nr, s2, n);
        }
    }
    if (k > 0) {
        if (nr > 0 && tc == 1) {
            if constexpr (std::is_same<T, float>::value)
                AFN_TRY(prod_tc(h->Wu2.as<float>(), k, nr, s2, n, zp, k, u, k, -1.f, 1.f, nrhs, part,
                                pcap, Bk, err, st));
        } else if (nr > 0 && tc == 2) {
            if constexpr (std::is_same<T, float>::value)
                AFN_TRY(prod_bf16(h->Wb2.as<__nv_bfloat16>(), k, nr, s2, n, zp, k, u, k, -1.f, 1.f,
                                  nrhs, part, pcap, Bk16, err, st));
        } else if (nr > 0) {
            prod<T, true, 0>(Wt, k, k, nr, s2, n, zp, k, u, k, (T)-1, (T)1, nrhs, part, pcap, st);
        } else {
            int64_t tot = k * nrhs;
            copy_cols_kernel<T><<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(zp, k, u, k, k, nrhs);
        }
        prod<T, false, 2>(LinvT, k, k, k, u, k, nullptr, 0, s1, n, (T)1, (T)0, nrhs, part, pcap, st);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "apply launch");
    return AFN_OK;
}

template afn_status afn_apply<float>(const Handle *, const float *, const float *, const float *,
                                     const float *, const float *, int, float *, float *,
                                     cudaStream_t);
template afn_status afn_apply<double>(const Handle *, const double *, const double *,
                                      const double *, const double *, const double *, int,
                                      double *, double *, cudaStream_t);

// ------------------------------------------------------- grouped apply --
// The apply of every member system of a group, one persistent launch per
// step of Alg. 3 (the same W-form as afn_apply), each over its own tile list:
//   zp  = L^{-1} r1                       (128-row blocks of k)
//   t   = r2 - W^T zp                     (128-row blocks of nr; t row-major)
//   y   = G t,  s2 = G^T y                (32-row blocks of nr, 8 lanes a row)
//   part_q = W[:, chunk q] s2[chunk q]    (128-row blocks of k x chunks)
//   u   = zp - sum_q part_q               (128-row blocks of k, chunks in order)
//   s1  = L^{-T} u
// r and s are the system's r32 and z32 (n x C column-major); a column group
// of 8 columns is the unit of every tile.

__device__ __forceinline__ bool group_live_ap(const GSys &S, int cg)
{
    const int c0 = cg * GC, c1 = min(S.nrhs, c0 + GC);
    for (int c = c0; c < c1; ++c)
        if (S.cs[c].active) return true;
    return false;
}

// MODE 0: zp = L^{-1} r1; 1: t = r2 - W^T zp; 2: W s2 partials; 3: s1 = L^{-T} u
template <int MODE>
__global__ void __launch_bounds__(256) gap_gemm_kernel(const GDev *__restrict__ gd)
{
    __shared__ __align__(16) float as[GK][GM + 4];
    __shared__ __align__(16) float xs[GK][GC + 4];
    const GTile *tiles = MODE == 1 ? gd->wb : (MODE == 2 ? gd->wtb : gd->kb);
    const int nt = MODE == 1 ? gd->nwb : (MODE == 2 ? gd->nwtb : gd->nkb);
    const int tc = threadIdx.x % 2, tr = threadIdx.x / 2;   // GemmShape<8>: TC = 2, RM = 1
    for (int ti = blockIdx.x; ti < nt; ti += gridDim.x) {
        const GTile tl = tiles[ti];
        const GSys &S = gd->sys[tl.sys];
        if (!group_live_ap(S, tl.cg)) continue;
        const int64_t n = S.n, k = S.k, nr = S.nr;
        const int C = S.ncg * GC;
        float acc[1][4];
        if (MODE == 0)
            gemm_rows<float, GC, false, 1>(S.Linv, k, k, tl.r0, 0, k, S.r32 + (int64_t)tl.cg * GC * n, n,
                                           as, xs, acc);
        else if (MODE == 1)
            gemm_rows<float, GC, false, 0>(S.Wt, k, nr, tl.r0, 0, k, S.zp + (int64_t)tl.cg * GC * k, k,
                                           as, xs, acc);
        else if (MODE == 2)
            gemm_rows<float, GC, true, 0>(S.Wt, k, k, tl.r0, (int64_t)tl.aux * S.kch,
                                          min(nr, (int64_t)(tl.aux + 1) * S.kch),
                                          S.z32 + (int64_t)tl.cg * GC * n + k, n, as, xs, acc);
        else
            gemm_rows<float, GC, false, 2>(S.LinvT, k, k, tl.r0, 0, k, S.u + (int64_t)tl.cg * GC * k, k,
                                           as, xs, acc);
        const int64_t gi = tl.r0 + tr;
        const int64_t M = MODE == 1 ? nr : k;
        if (gi >= M) continue;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int c = tl.cg * GC + tc * 4 + b;
            const float v = acc[0][b];
            if (MODE == 0) S.zp[(int64_t)c * k + gi] = v;
            else if (MODE == 1)
                S.t[((int64_t)tl.cg * nr + gi) * GC + tc * 4 + b] = S.r32[(int64_t)c * n + k + gi] - v;
            else if (MODE == 2) S.part[((int64_t)tl.aux * C + c) * k + gi] = v;
            else S.z32[(int64_t)c * n + gi] = v;
        }
    }
}

// u = zp - sum_q part_q, chunks in order
__global__ void __launch_bounds__(256) gap_finish_kernel(const GDev *__restrict__ gd)
{
    const int nt = gd->nkb;
    for (int ti = blockIdx.x; ti < nt; ti += gridDim.x) {
        const GTile tl = gd->kb[ti];
        const GSys &S = gd->sys[tl.sys];
        if (!group_live_ap(S, tl.cg)) continue;
        const int64_t k = S.k;
        const int C = S.ncg * GC;
        for (int e = threadIdx.x; e < GM * GC; e += 256) {
            const int64_t i = tl.r0 + e % GM;
            const int c = tl.cg * GC + e / GM;
            if (i >= k) continue;
            float v = S.zp[(int64_t)c * k + i];
            for (int q = 0; q < S.js; ++q) v -= S.part[((int64_t)q * C + c) * k + i];
            S.u[(int64_t)c * k + i] = v;
        }
    }
}

// MODE 0: y = G t (ELL rows); 1: s2 = G^T y (CSR of G^T).  8 lanes per row,
// lane = column of the group; t and y are row-major [nr][8].
template <int MODE>
__global__ void __launch_bounds__(256) gap_sparse_kernel(const GDev *__restrict__ gd)
{
    const int nt = gd->nsp;
    const int c = threadIdx.x % GC;
    for (int ti = blockIdx.x; ti < nt; ti += gridDim.x) {
        const GTile tl = gd->sp[ti];
        const GSys &S = gd->sys[tl.sys];
        if (!group_live_ap(S, tl.cg)) continue;
        const int64_t nr = S.nr;
        const int64_t i = tl.r0 + threadIdx.x / GC;
        if (i >= nr) continue;
        float acc = 0.f;
        if (MODE == 0) {
            const float *t = S.t + (int64_t)tl.cg * nr * GC;
            const int w = S.w;
            for (int p = 0; p < w; ++p) {
                const int32_t j = S.pat[i * w + p];
                if (j < 0) break;
                acc += S.G[i * w + p] * t[(int64_t)j * GC + c];
            }
            S.y[((int64_t)tl.cg * nr + i) * GC + c] = acc;
        } else {
            const float *y = S.y + (int64_t)tl.cg * nr * GC;
            const int32_t q0 = S.gptr[i], q1 = S.gptr[i + 1];
            for (int32_t q = q0; q < q1; ++q) acc += S.G[S.gslot[q]] * y[(int64_t)S.grow[q] * GC + c];
            S.z32[((int64_t)tl.cg * GC + c) * S.n + S.k + i] = acc;
        }
    }
}

int group_sparse_rows() { return 256 / GC; }
int group_block_rows() { return GM; }

afn_status group_apply(const GDev *gd, cudaStream_t s, double share, int cps)
{
    const int g = persistent_grid(cps > 0 ? cps : 4, share);
    gap_gemm_kernel<0><<<g, 256, 0, s>>>(gd);
    gap_gemm_kernel<1><<<g, 256, 0, s>>>(gd);
    gap_sparse_kernel<0><<<g, 256, 0, s>>>(gd);
    gap_sparse_kernel<1><<<g, 256, 0, s>>>(gd);
    gap_gemm_kernel<2><<<g, 256, 0, s>>>(gd);
    gap_finish_kernel<<<g, 256, 0, s>>>(gd);
    gap_gemm_kernel<3><<<g, 256, 0, s>>>(gd);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? AFN_OK : cuda_fail(e, "grouped apply launch");
}

}  // namespace afn
