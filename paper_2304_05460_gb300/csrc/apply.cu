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
#include <algorithm>

#include "afn_device.cuh"
#include "afn_internal.cuh"

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

// out[i,c] = y[i,c] - sum_js part[js][c][i]
template <class T>
__global__ void colmul_finish(const T *__restrict__ part, int js, int nc, int64_t ncols,
                              const T *__restrict__ Y, int64_t ldy, T *__restrict__ O,
                              int64_t ldo)
{
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= ncols * nc) return;
    int c = (int)(e / ncols);
    int64_t i = e % ncols;
    T s = 0;
    for (int q = 0; q < js; ++q) s += part[((int64_t)q * nc + c) * ncols + i];
    O[c * ldo + i] = Y[c * ldy + i] - s;
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

size_t apply_tmp_elems(const Handle *h, int nrhs)
{
    int64_t k = h->k, nr = h->nr;
    int js = colmul_js(nr, k);
    int piece_max = 16;
    return (size_t)(2 * k * nrhs + 2 * nr * nrhs) + (size_t)js * piece_max * (size_t)std::max<int64_t>(k, 1) + 64;
}

template <class T>
afn_status afn_apply(const Handle *h, const T *Linv, const T *LinvT, const T *Wt, const T *G,
                     const T *r, int nrhs, T *s, T *tmp, cudaStream_t st)
{
    const int64_t n = h->n, k = h->k, nr = h->nr;
    const int w = h->w;
    T *zp = tmp;                       // k x nrhs
    T *u = zp + k * nrhs;              // k x nrhs
    T *t = u + k * nrhs;               // nr x nrhs
    T *y = t + nr * nrhs;              // nr x nrhs
    T *part = y + nr * nrhs;           // js x 16 x k
    const T *r1 = r, *r2 = r + k;
    T *s1 = s, *s2 = s + k;
    if (k > 0) rowmul<T, 1>(Linv, k, k, k, r1, n, nullptr, 0, zp, k, (T)1, (T)0, nrhs, st);
    if (nr > 0) {
        if (k > 0) rowmul<T, 0>(Wt, k, nr, k, zp, k, r2, n, t, nr, (T)-1, (T)1, nrhs, st);
        else {
            int64_t tot = nr * nrhs;
            copy_cols_kernel<T><<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(r2, n, t, nr, nr, nrhs);
        }
        int64_t tot = nr * nrhs;
        unsigned g = (unsigned)((tot + 255) / 256);
        spmv_ell_kernel<T><<<g, 256, 0, st>>>(G, h->pat.as<int32_t>(), nr, w, nrhs, t, nr, y, nr);
        spmv_gt_kernel<T><<<g, 256, 0, st>>>(G, h->gt_ptr.as<int32_t>(), h->gt_row.as<int32_t>(),
                                             h->gt_slot.as<int32_t>(), nr, nrhs, y, nr, s2, n);
    }
    if (k > 0) {
        if (nr > 0) {
            int js = colmul_js(nr, k);
            int64_t chunk = (nr + js - 1) / js;
            js = (int)((nr + chunk - 1) / chunk);
            for (int c0 = 0; c0 < nrhs;) {
                int b = piece(nrhs - c0, 16);
                dim3 grid((unsigned)((k + CT - 1) / CT), (unsigned)js);
                const T *x = s2 + c0 * n;
                switch (b) {
                case 1: colmul_kernel<T, 1><<<grid, CT, 0, st>>>(Wt, k, nr, k, x, n, part, chunk); break;
                case 2: colmul_kernel<T, 2><<<grid, CT, 0, st>>>(Wt, k, nr, k, x, n, part, chunk); break;
                case 4: colmul_kernel<T, 4><<<grid, CT, 0, st>>>(Wt, k, nr, k, x, n, part, chunk); break;
                case 8: colmul_kernel<T, 8><<<grid, CT, 0, st>>>(Wt, k, nr, k, x, n, part, chunk); break;
                default: colmul_kernel<T, 16><<<grid, CT, 0, st>>>(Wt, k, nr, k, x, n, part, chunk); break;
                }
                int64_t tot = k * b;
                colmul_finish<T><<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(
                    part, js, b, k, zp + c0 * k, k, u + c0 * k, k);
                c0 += b;
            }
        } else {
            int64_t tot = k * nrhs;
            copy_cols_kernel<T><<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(zp, k, u, k, k, nrhs);
        }
        rowmul<T, 2>(LinvT, k, k, k, u, k, nullptr, 0, s1, n, (T)1, (T)0, nrhs, st);
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

}  // namespace afn
