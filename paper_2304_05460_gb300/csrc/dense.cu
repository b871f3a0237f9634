// dense.cu -- dense pieces of the AFN build (Alg. 2):
//   * kernel blocks K(X_a, X_b) (K11 + mu I, K12),
//   * the blocked right-looking Cholesky of K11 + mu I in FP64,
//   * L^{-1} by recursive doubling in FP64: 64 x 64 diagonal blocks inverted
//     by substitution, then per level the lower-left block -C^{-1} B A^{-1} of
//     every 2b-block as batched triangular GEMMs (rounded once to FP32 for
//     mixed handles),
//   * W^T = K12^T L^{-T} as one tiled GEMM that skips the triangular
//     operand's zero tiles (FP64, FP32, or double-float on the FP32 pipes for
//     DF handles),
//   * the blocked solve B <- B L^{-T} (the Nystrom factor B = K(X, X_S) L^{-T}),
// all on row-major storage.
#include <algorithm>
#include <cmath>

#include "afn_device.cuh"
#include "afn_internal.cuh"

namespace afn {

// ------------------------------------------------------------ kernel block --
// out[i*ld + j] = K(a_i, b_j) (+ shift when i == j), FP64, the definition of
// eq. (gaussianf) / Sec. 5 on an exact squared distance.
__global__ void kernel_block_kernel(const double *__restrict__ Xa, int64_t na,
                                    const double *__restrict__ Xb, int64_t nb, int d, int kernel,
                                    double l, double shift, double *__restrict__ out, int64_t ld)
{
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= na * nb) return;
    int64_t i = e / nb, j = e % nb;
    double r2 = sqdist_exact(Xa + i * d, Xb + j * d, d);
    double v = kernel64(r2, kernel, l);
    if (i == j) v += shift;
    out[i * ld + j] = v;
}

afn_status kernel_block(const double *Xa, int64_t na, const double *Xb, int64_t nb, int d,
                        KParams kp, double diag_shift, double *out, int64_t ld, cudaStream_t s)
{
    int64_t tot = na * nb;
    if (tot == 0) return AFN_OK;
    kernel_block_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(Xa, na, Xb, nb, d, kp.kernel,
                                                                       kp.l, diag_shift, out, ld);
    AFN_CUDA(cudaGetLastError());
    return AFN_OK;
}

// FP32 kernel block on prescaled points (stored dims ds): out[i*ld+j]
template <int KER>
__global__ void kernel_block32_kernel(const float *__restrict__ Xa, int64_t na,
                                      const float *__restrict__ Xb, int64_t nb, int ds,
                                      float *__restrict__ out, int64_t ld)
{
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= na * nb) return;
    int64_t i = e / nb, j = e % nb;
    float r2 = 0.f;
    for (int t = 0; t < ds; ++t) {
        float u = Xa[i * ds + t] - Xb[j * ds + t];
        r2 = fmaf(u, u, r2);
    }
    out[i * ld + j] = kernel32_scaled<KER>(r2);
}

afn_status kernel_block32(const float *Xa, int64_t na, const float *Xb, int64_t nb, int dp,
                          int kernel, float *out, int64_t ld, cudaStream_t s)
{
    int64_t tot = na * nb;
    if (tot == 0) return AFN_OK;
    int ds = dp == 3 ? 4 : dp;
    unsigned g = (unsigned)((tot + 255) / 256);
    if (kernel == 0) kernel_block32_kernel<0><<<g, 256, 0, s>>>(Xa, na, Xb, nb, ds, out, ld);
    else kernel_block32_kernel<1><<<g, 256, 0, s>>>(Xa, na, Xb, nb, ds, out, ld);
    AFN_CUDA(cudaGetLastError());
    return AFN_OK;
}

// ---------------------------------------------------------------- Cholesky --
static constexpr int NB = 32;   // panel width

// factor the nb x nb diagonal block at (kb, kb) in shared memory
// tiny < 0: a pivot <= 0 flags DEV_NOT_SPD; tiny >= 0: a pivot <= tiny is
// treated as zero (its column of L is zero: the point is already spanned).
__global__ void potrf_diag_kernel(double *A, int64_t k, int64_t kb, int nb, int *status,
                                  double tiny)
{
    __shared__ double a[NB][NB + 1];
    for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
        int r = e / nb, c = e % nb;
        a[r][c] = (c <= r) ? A[(kb + r) * k + kb + c] : 0.0;
    }
    __syncthreads();
    for (int j = 0; j < nb; ++j) {
        __shared__ double piv;
        if (threadIdx.x == 0) {
            double v = a[j][j];
            if (tiny >= 0.0) {
                piv = (v > tiny) ? sqrt(v) : 0.0;
            } else {
                if (!(v > 0.0)) {
                    atomicExch(status, DEV_NOT_SPD);
                    v = 1.0;
                }
                piv = sqrt(v);
            }
            a[j][j] = piv;
        }
        __syncthreads();
        for (int r = j + 1 + threadIdx.x; r < nb; r += blockDim.x)
            a[r][j] = (piv != 0.0) ? a[r][j] / piv : 0.0;
        __syncthreads();
        for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
            int r = e / nb, c = e % nb;
            if (c > j && r >= c) a[r][c] -= a[r][j] * a[c][j];
        }
        __syncthreads();
    }
    for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
        int r = e / nb, c = e % nb;
        A[(kb + r) * k + kb + c] = (c <= r) ? a[r][c] : 0.0;
    }
}

// rows below the diagonal block: A[r, kb:kb+nb] <- A[r, kb:kb+nb] L_bb^{-T}
template <class T>
__global__ void trsm_rows_kernel(const T *__restrict__ Lsrc, int64_t ldl, int64_t lb,
                                 T *__restrict__ B, int64_t ldb, int64_t r0, int64_t m,
                                 int64_t cb, int nb)
{
    __shared__ T lbb[NB][NB + 1];
    __shared__ T xs[128][NB + 1];
    for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
        int r = e / nb, c = e % nb;
        lbb[r][c] = Lsrc[(lb + r) * ldl + lb + c];
    }
    int64_t row = r0 + (int64_t)blockIdx.x * 128 + threadIdx.x;
    __syncthreads();
    if (row >= m) return;
    T *b = B + row * ldb + cb;
    for (int c = 0; c < nb; ++c) {
        T v = b[c];
        for (int p = 0; p < c; ++p) v -= xs[threadIdx.x][p] * lbb[c][p];
        xs[threadIdx.x][c] = (lbb[c][c] != (T)0) ? v / lbb[c][c] : (T)0;
    }
    for (int c = 0; c < nb; ++c) b[c] = xs[threadIdx.x][c];
}

// C[m x nb] -= A[m x K] * Bm[nb x K]^T   (C = B[:, cb:cb+nb], A = B[:, 0:K],
// Bm = L[cb:cb+nb, 0:K]); 128-row tiles, 256 threads, 4 rows x 4 cols each.
template <class T>
__global__ void __launch_bounds__(256) gemm_nt_update_kernel(const T *__restrict__ A, int64_t lda,
                                                             const T *__restrict__ Bm,
                                                             int64_t ldbm, T *__restrict__ C,
                                                             int64_t ldc, int64_t m, int nb,
                                                             int64_t K)
{
    constexpr int TM = 128, KC = 16;
    __shared__ T as[KC][TM + 1];
    __shared__ T bs[KC][NB + 1];
    const int tx = threadIdx.x % 8;    // column group: cols tx*4..+3
    const int ty = threadIdx.x / 8;    // row group: rows ty*4..+3
    const int64_t r0 = (int64_t)blockIdx.x * TM;
    T acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = 0;
    for (int64_t k0 = 0; k0 < K; k0 += KC) {
        __syncthreads();
        for (int e = threadIdx.x; e < TM * KC; e += 256) {
            int r = e / KC, kk = e % KC;
            int64_t gr = r0 + r, gk = k0 + kk;
            as[kk][r] = (gr < m && gk < K) ? A[gr * lda + gk] : (T)0;
        }
        for (int e = threadIdx.x; e < NB * KC; e += 256) {
            int c = e / KC, kk = e % KC;
            int64_t gk = k0 + kk;
            bs[kk][c] = (c < nb && gk < K) ? Bm[(int64_t)c * ldbm + gk] : (T)0;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < KC; ++kk) {
            T av[4], bv[4];
#pragma unroll
            for (int a = 0; a < 4; ++a) av[a] = as[kk][ty * 4 + a];
#pragma unroll
            for (int b = 0; b < 4; ++b) bv[b] = bs[kk][tx * 4 + b];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) acc[a][b] += av[a] * bv[b];
        }
    }
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        int64_t gr = r0 + ty * 4 + a;
        if (gr >= m) continue;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            int c = tx * 4 + b;
            if (c < nb) C[gr * ldc + c] -= acc[a][b];
        }
    }
}

// trailing update of the Cholesky: A[r, c] -= sum_p A[r, kb+p] A[c, kb+p]
// for kb+nb <= c <= r < k (64 x 64 lower tiles)
__global__ void __launch_bounds__(256) syrk_update_kernel(double *A, int64_t k, int64_t kb, int nb)
{
    const int64_t t0 = kb + nb;
    const int64_t ti = blockIdx.y, tj = blockIdx.x;
    if (tj > ti) return;
    const int64_t r0 = t0 + ti * 64, c0 = t0 + tj * 64;
    __shared__ double pr[NB][65];
    __shared__ double pc[NB][65];
    for (int e = threadIdx.x; e < 64 * NB; e += 256) {
        int r = e / NB, p = e % NB;
        int64_t gr = r0 + r, gc = c0 + r;
        pr[p][r] = (gr < k && p < nb) ? A[gr * k + kb + p] : 0.0;
        pc[p][r] = (gc < k && p < nb) ? A[gc * k + kb + p] : 0.0;
    }
    __syncthreads();
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    double acc[4][4] = {};
    for (int p = 0; p < nb; ++p) {
        double a[4], b[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) { a[q] = pr[p][ty * 4 + q]; b[q] = pc[p][tx * 4 + q]; }
#pragma unroll
        for (int x = 0; x < 4; ++x)
#pragma unroll
            for (int y = 0; y < 4; ++y) acc[x][y] += a[x] * b[y];
    }
#pragma unroll
    for (int x = 0; x < 4; ++x) {
        int64_t gr = r0 + ty * 4 + x;
        if (gr >= k) continue;
#pragma unroll
        for (int y = 0; y < 4; ++y) {
            int64_t gc = c0 + tx * 4 + y;
            if (gc < k && gc <= gr) A[gr * k + gc] -= acc[x][y];
        }
    }
}

__global__ void zero_upper_kernel(double *A, int64_t k)
{
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= k * k) return;
    int64_t r = e / k, c = e % k;
    if (c > r) A[e] = 0.0;
}

afn_status cholesky64(double *A, int64_t k, int *status, cudaStream_t s, double tiny)
{
    if (k <= 0) return AFN_OK;
    if (k > 65535 * 64) {
        set_error("cholesky: k=%lld too large", (long long)k);
        return AFN_ERR_ARG;
    }
    AFN_CUDA(cudaMemsetAsync(status, 0, sizeof(int), s));
    for (int64_t kb = 0; kb < k; kb += NB) {
        int nb = (int)std::min<int64_t>(NB, k - kb);
        potrf_diag_kernel<<<1, 256, 0, s>>>(A, k, kb, nb, status, tiny);
        int64_t below = k - kb - nb;
        if (below > 0) {
            trsm_rows_kernel<double><<<(unsigned)((below + 127) / 128), 128, 0, s>>>(
                A, k, kb, A, k, kb + nb, k, kb, nb);
            unsigned T = (unsigned)((below + 63) / 64);
            syrk_update_kernel<<<dim3(T, T), 256, 0, s>>>(A, k, kb, nb);
        }
    }
    zero_upper_kernel<<<(unsigned)((k * k + 255) / 256), 256, 0, s>>>(A, k);
    AFN_CUDA(cudaGetLastError());
    return AFN_OK;
}

// ------------------------------------------------------------------ TRSM --
// B (m x k row-major) <- B L^{-T}, L (k x k lower row-major):
// left-looking over panels of NB columns:
//   B[:, P] -= B[:, 0:p0] L[P, 0:p0]^T ;  B[:, P] <- B[:, P] L[P,P]^{-T}
template <class T>
static afn_status trsm_right_lt(const T *L, int64_t k, T *B, int64_t m, cudaStream_t s)
{
    if (k <= 0 || m <= 0) return AFN_OK;
    for (int64_t p0 = 0; p0 < k; p0 += NB) {
        int nb = (int)std::min<int64_t>(NB, k - p0);
        if (p0 > 0) {
            gemm_nt_update_kernel<T><<<(unsigned)((m + 127) / 128), 256, 0, s>>>(
                B, k, L + p0 * k, k, B + p0, k, m, nb, p0);
        }
        trsm_rows_kernel<T><<<(unsigned)((m + 127) / 128), 128, 0, s>>>(L, k, p0, B, k, 0, m, p0, nb);
    }
    AFN_CUDA(cudaGetLastError());
    return AFN_OK;
}

afn_status trsm_right_lt64(const double *L, int64_t k, double *B, int64_t m, cudaStream_t s)
{
    return trsm_right_lt<double>(L, k, B, m, s);
}



template <class T>
__global__ void transpose_kernel(const T *__restrict__ A, int64_t k, T *__restrict__ B)
{
    __shared__ T t[32][33];
    int64_t bx = (int64_t)blockIdx.x * 32, by = (int64_t)blockIdx.y * 32;
    for (int q = threadIdx.y; q < 32; q += blockDim.y) {
        int64_t r = by + q, c = bx + threadIdx.x;
        if (r < k && c < k) t[q][threadIdx.x] = A[r * k + c];
    }
    __syncthreads();
    for (int q = threadIdx.y; q < 32; q += blockDim.y) {
        int64_t r = bx + q, c = by + threadIdx.x;
        if (r < k && c < k) B[r * k + c] = t[threadIdx.x][q];
    }
}


// ------------------------------------------------------------------ GEMM --
// C = alpha A B on the CUDA cores, A (M x K), B (K x N), C (M x N), all
// row-major with leading dimensions; batch z adds z * (sa, sb, sc) to the
// three pointers.  MODE says which operand is triangular, so a tile reads only
// the K-range where both operands can be nonzero:
//   GM_B_UPPER  B[q][p] = 0 for q > p  (column tile [n0, n0 + BN): q < n0 + BN)
//   GM_B_LOWER  B[q][p] = 0 for q < p  (q >= n0)
//   GM_A_LOWER  A[m][q] = 0 for q > m  (row tile [m0, m0 + BM): q < m0 + BM)
// The zeros inside the range are read as stored.  Each output is the sum over
// q in ascending order.  FP32: 128 x 128 tiles, 8 x 8 outputs per thread;
// FP64: 64 x 64 tiles, 4 x 4 per thread (GB300 retires few FP64 FMAs per
// cycle, so the tile only needs enough reuse to keep that pipe busy).  8-deep
// K slices double-buffered in shared memory.
enum : int { GM_B_UPPER = 1, GM_B_LOWER = 2, GM_A_LOWER = 4 };

template <class T> struct GemmTile;
template <> struct GemmTile<float> { static constexpr int B = 128, R = 8; };
template <> struct GemmTile<double> { static constexpr int B = 64, R = 4; };

template <class T, int MODE>
__global__ void __launch_bounds__(256) gemm_tri_kernel(const T *__restrict__ A, int64_t lda, int64_t sa,
                                                       const T *__restrict__ B, int64_t ldb, int64_t sb,
                                                       T *__restrict__ C, int64_t ldc, int64_t sc,
                                                       int64_t M, int64_t N, int64_t K, T alpha)
{
    constexpr int BT = GemmTile<T>::B, R = GemmTile<T>::R, BK = 8;
    constexpr int H = BT / 2;                       // outputs of a thread: rows {ty R/2 + i, H + ...}
    constexpr int LA = BT * BK / 256;               // A elements loaded per thread per slice
    __shared__ __align__(16) T As[2][BK][BT];
    __shared__ __align__(16) T Bs[2][BK][BT];
    A += (int64_t)blockIdx.z * sa;
    B += (int64_t)blockIdx.z * sb;
    C += (int64_t)blockIdx.z * sc;
    const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
    const int64_t m0 = (int64_t)blockIdx.y * BT, n0 = (int64_t)blockIdx.x * BT;
    int64_t klo = (MODE & GM_B_LOWER) ? n0 : 0, khi = K;
    if (MODE & GM_B_UPPER) khi = min(khi, n0 + BT);
    if (MODE & GM_A_LOWER) khi = min(khi, m0 + BT);
    // this thread's loads: A row m0 + tid / (BK / LA), K-elements (tid % (BK / LA)) LA + u;
    // B row tid / 32 of the slice, columns (tid % 32) LA + u
    const int am = tid / (BK / LA), ak = (tid % (BK / LA)) * LA;
    const int bk = tid / 32, bn = (tid % 32) * LA;
    T ra[LA], rb[LA];
    auto fetch = [&](int64_t k0) {
#pragma unroll
        for (int u = 0; u < LA; ++u) {
            const int64_t gm = m0 + am, gk = k0 + ak + u;
            ra[u] = (gm < M && gk < khi) ? A[gm * lda + gk] : (T)0;
            const int64_t gq = k0 + bk, gp = n0 + bn + u;
            rb[u] = (gq < khi && gp < N) ? B[gq * ldb + gp] : (T)0;
        }
    };
    auto stash = [&](int buf) {
#pragma unroll
        for (int u = 0; u < LA; ++u) {
            As[buf][ak + u][am] = ra[u];
            Bs[buf][bk][bn + u] = rb[u];
        }
    };
    T acc[R][R];
#pragma unroll
    for (int i = 0; i < R; ++i)
#pragma unroll
        for (int j = 0; j < R; ++j) acc[i][j] = (T)0;
    const int nt = khi > klo ? (int)((khi - klo + BK - 1) / BK) : 0;
    if (nt > 0) {
        fetch(klo);
        stash(0);
    }
    __syncthreads();
    for (int t = 0; t < nt; ++t) {
        const int buf = t & 1;
        if (t + 1 < nt) fetch(klo + (int64_t)(t + 1) * BK);
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            T av[R], bv[R];
#pragma unroll
            for (int i = 0; i < R / 2; ++i) {
                av[i] = As[buf][kk][ty * (R / 2) + i];
                av[R / 2 + i] = As[buf][kk][H + ty * (R / 2) + i];
                bv[i] = Bs[buf][kk][tx * (R / 2) + i];
                bv[R / 2 + i] = Bs[buf][kk][H + tx * (R / 2) + i];
            }
#pragma unroll
            for (int i = 0; i < R; ++i)
#pragma unroll
                for (int j = 0; j < R; ++j) acc[i][j] = fma(av[i], bv[j], acc[i][j]);
        }
        if (t + 1 < nt) stash(buf ^ 1);     // the other buffer was last read before the previous barrier
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < R; ++i) {
        const int64_t gm = m0 + (i < R / 2 ? ty * (R / 2) + i : H + ty * (R / 2) + (i - R / 2));
        if (gm >= M) continue;
#pragma unroll
        for (int j = 0; j < R; ++j) {
            const int64_t gp = n0 + (j < R / 2 ? tx * (R / 2) + j : H + tx * (R / 2) + (j - R / 2));
            if (gp < N) C[gm * ldc + gp] = alpha * acc[i][j];
        }
    }
}

template <class T, int MODE>
static void gemm_tri(const T *A, int64_t lda, int64_t sa, const T *B, int64_t ldb, int64_t sb, T *C,
                     int64_t ldc, int64_t sc, int64_t M, int64_t N, int64_t K, T alpha, int batch,
                     cudaStream_t s)
{
    constexpr int BT = GemmTile<T>::B;
    if (M <= 0 || N <= 0 || batch <= 0) return;
    dim3 g((unsigned)((N + BT - 1) / BT), (unsigned)((M + BT - 1) / BT), (unsigned)batch);
    gemm_tri_kernel<T, MODE><<<g, 256, 0, s>>>(A, lda, sa, B, ldb, sb, C, ldc, sc, M, N, K, alpha);
}

// Inverses of the 64 x 64 diagonal blocks of L (one CTA per block, one thread
// per column: forward substitution of the unit vector, p ascending).
static constexpr int TI_B = 64;

template <class T>
__global__ void __launch_bounds__(TI_B) diag_inverse_kernel(const T *__restrict__ L, int64_t k,
                                                            T *__restrict__ Linv)
{
    // dynamic shared memory: lb[TI_B][TI_B + 1] (the block of L), then
    // xs[TI_B][TI_B + 1] (xs[i][c]: row i of column c of the block inverse)
    extern __shared__ __align__(16) unsigned char tism[];
    T(*lb)[TI_B + 1] = reinterpret_cast<T(*)[TI_B + 1]>(tism);
    T(*xs)[TI_B + 1] = reinterpret_cast<T(*)[TI_B + 1]>(tism + sizeof(T) * TI_B * (TI_B + 1));
    const int64_t r0 = (int64_t)blockIdx.x * TI_B;
    const int nb = (int)(k - r0 < TI_B ? k - r0 : TI_B);
    for (int e = threadIdx.x; e < nb * nb; e += TI_B) {
        const int r = e / nb, c = e % nb;
        lb[r][c] = L[(r0 + r) * k + r0 + c];
    }
    __syncthreads();
    const int c = threadIdx.x;
    if (c >= nb) return;
    for (int i = c; i < nb; ++i) {
        T v = (i == c) ? (T)1 : (T)0;
        for (int p = c; p < i; ++p) v -= lb[i][p] * xs[p][c];
        xs[i][c] = v / lb[i][i];
        Linv[(r0 + i) * k + r0 + c] = xs[i][c];
    }
}

// Linv = L^{-1} (lower, row-major) by recursive doubling over block sizes
// b = 64, 128, ...: with [A 0; B C] the 2b-block at i0 (A, C already
// inverted), its lower-left block is -C^{-1} (B A^{-1}); the products run as
// batched tiled GEMMs over all 2b-blocks of a level (the one at the end of
// the matrix, which may be shorter, in its own launch).  LinvT holds
// T = B A^{-1} during the levels and L^{-T} at the end.
template <class T>
static afn_status tri_inverse(const T *L, int64_t k, T *Linv, T *LinvT, cudaStream_t s)
{
    if (k <= 0) return AFN_OK;
    AFN_CUDA(cudaMemsetAsync(Linv, 0, sizeof(T) * (size_t)(k * k), s));
    const int dsm = (int)(2 * sizeof(T) * TI_B * (TI_B + 1));
    cudaFuncSetAttribute(diag_inverse_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, dsm);
    diag_inverse_kernel<T><<<(unsigned)((k + TI_B - 1) / TI_B), TI_B, dsm, s>>>(L, k, Linv);
    for (int64_t b = TI_B; b < k; b *= 2) {
        const int64_t st = 2 * b * k + 2 * b;                // one 2b-block further down the diagonal
        const int64_t full = (k - b) / (2 * b);              // pairs whose C block has b rows
        const int64_t i0l = full * 2 * b;                    // the pair at the end, if any
        const int64_t cl = i0l + b < k ? std::min<int64_t>(b, k - i0l - b) : 0;
        auto level = [&](int64_t i0, int64_t c, int batch) {
            const int64_t a = i0 * k + i0, bl = (i0 + b) * k + i0, cc = (i0 + b) * k + i0 + b;
            // T = B A^{-1}   (A^{-1} lower triangular)
            gemm_tri<T, GM_B_LOWER>(L + bl, k, st, Linv + a, k, st, LinvT + bl, k, st, c, b, b,
                                    (T)1, batch, s);
            // lower-left block = -C^{-1} T   (C^{-1} lower triangular)
            gemm_tri<T, GM_A_LOWER>(Linv + cc, k, st, LinvT + bl, k, st, Linv + bl, k, st, c, b, c,
                                    (T)-1, batch, s);
        };
        if (full > 0 && i0l + b < k && cl == b) {
            level(0, b, (int)(full + 1));
        } else {
            if (full > 0) level(0, b, (int)full);
            if (cl > 0) level(i0l, cl, 1);
        }
    }
    dim3 gt((unsigned)((k + 31) / 32), (unsigned)((k + 31) / 32));
    transpose_kernel<T><<<gt, dim3(32, 8), 0, s>>>(Linv, k, LinvT);
    AFN_CUDA(cudaGetLastError());
    return AFN_OK;
}

afn_status tri_inverse64(const double *L, int64_t k, double *Linv, double *LinvT, cudaStream_t s)
{
    return tri_inverse<double>(L, k, Linv, LinvT, s);
}


// The same product with FP64 operands and result but double-float arithmetic
// on the FP32 pipes (GB300 retires about 64 FP32 operations per FP64 one):
// each operand is split on staging into hi + lo floats (hi = float(x), lo =
// float(x - hi)), each product term is formed exactly by the FMA-based
// TwoProduct of the hi parts plus the two cross terms (Dekker 1971), and
// the running sum is a double-float (Knuth's TwoSum on the high parts, the
// low parts added); the result is hi + lo in FP64.  Relative error about
// K 2^-48 of sum |a b|, for the W products of double-float handles.
static constexpr int DF_B = 64, DF_BK = 8;

__global__ void __launch_bounds__(256) dfgemm_upper_kernel(const double *__restrict__ A, int64_t lda,
                                                           const double *__restrict__ B, int64_t ldb,
                                                           double *__restrict__ C, int64_t ldc,
                                                           int64_t M, int64_t N, int64_t K)
{
    __shared__ __align__(16) float Ah[2][DF_BK][DF_B], Al[2][DF_BK][DF_B];
    __shared__ __align__(16) float Bh[2][DF_BK][DF_B], Bl[2][DF_BK][DF_B];
    const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
    const int64_t m0 = (int64_t)blockIdx.y * DF_B, n0 = (int64_t)blockIdx.x * DF_B;
    const int64_t khi = min(K, n0 + DF_B);              // B upper triangular
    const int am = tid / 4, ak = (tid % 4) * 2;
    const int bk = tid / 32, bn = (tid % 32) * 2;
    double ra[2], rb[2];
    auto fetch = [&](int64_t k0) {
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int64_t gm = m0 + am, gk = k0 + ak + u;
            ra[u] = (gm < M && gk < khi) ? A[gm * lda + gk] : 0.0;
            const int64_t gq = k0 + bk, gp = n0 + bn + u;
            rb[u] = (gq < khi && gp < N) ? B[gq * ldb + gp] : 0.0;
        }
    };
    auto stash = [&](int buf) {
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const float ah = (float)ra[u], bh = (float)rb[u];
            Ah[buf][ak + u][am] = ah;
            Al[buf][ak + u][am] = (float)(ra[u] - (double)ah);
            Bh[buf][bk][bn + u] = bh;
            Bl[buf][bk][bn + u] = (float)(rb[u] - (double)bh);
        }
    };
    float sh[4][4], sl[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) sh[i][j] = sl[i][j] = 0.f;
    const int nt = (int)((khi + DF_BK - 1) / DF_BK);
    if (nt > 0) {
        fetch(0);
        stash(0);
    }
    __syncthreads();
    for (int t = 0; t < nt; ++t) {
        const int buf = t & 1;
        if (t + 1 < nt) fetch((int64_t)(t + 1) * DF_BK);
#pragma unroll
        for (int kk = 0; kk < DF_BK; ++kk) {
            float ah[4], al[4], bh[4], bl[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                ah[i] = Ah[buf][kk][ty * 4 + i];
                al[i] = Al[buf][kk][ty * 4 + i];
                bh[i] = Bh[buf][kk][tx * 4 + i];
                bl[i] = Bl[buf][kk][tx * 4 + i];
            }
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const float p = __fmul_rn(ah[i], bh[j]);
                    float e = __fmaf_rn(ah[i], bh[j], -p);
                    e = __fmaf_rn(ah[i], bl[j], e);
                    e = __fmaf_rn(al[i], bh[j], e);
                    const float s1 = __fadd_rn(sh[i][j], p);
                    const float bb = __fsub_rn(s1, sh[i][j]);
                    const float err = __fadd_rn(__fsub_rn(sh[i][j], __fsub_rn(s1, bb)), __fsub_rn(p, bb));
                    sh[i][j] = s1;
                    sl[i][j] = __fadd_rn(sl[i][j], __fadd_rn(err, e));
                }
        }
        if (t + 1 < nt) stash(buf ^ 1);
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int64_t gm = m0 + ty * 4 + i;
        if (gm >= M) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int64_t gp = n0 + tx * 4 + j;
            if (gp < N) C[gm * ldc + gp] = (double)sh[i][j] + (double)sl[i][j];
        }
    }
}

afn_status gemm_upper_df(const double *A, int64_t m, int64_t k, const double *U, double *C, cudaStream_t s)
{
    if (m <= 0 || k <= 0) return AFN_OK;
    dim3 g((unsigned)((k + DF_B - 1) / DF_B), (unsigned)((m + DF_B - 1) / DF_B));
    dfgemm_upper_kernel<<<g, 256, 0, s>>>(A, k, U, k, C, k, m, k, k);
    AFN_CUDA(cudaGetLastError());
    return AFN_OK;
}

// C (m x k) = A (m x k) U with U (k x k) upper triangular, FP64, row-major
afn_status gemm_upper64(const double *A, int64_t m, int64_t k, const double *U, double *C, cudaStream_t s)
{
    if (m <= 0 || k <= 0) return AFN_OK;
    gemm_tri<double, GM_B_UPPER>(A, k, 0, U, k, 0, C, k, 0, m, k, k, 1.0, 1, s);
    AFN_CUDA(cudaGetLastError());
    return AFN_OK;
}

// C (m x k) = A (m x k) U with U (k x k) upper triangular, FP32, row-major
afn_status gemm_upper32(const float *A, int64_t m, int64_t k, const float *U, float *C, cudaStream_t s)
{
    if (m <= 0 || k <= 0) return AFN_OK;
    gemm_tri<float, GM_B_UPPER>(A, k, 0, U, k, 0, C, k, 0, m, k, k, 1.f, 1, s);
    AFN_CUDA(cudaGetLastError());
    return AFN_OK;
}

// ------------------------------------------------------------- conversion --
__global__ void cvt64to32_kernel(const double *__restrict__ a, float *__restrict__ b, int64_t n)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = (float)a[i];
}

__global__ void cvt32to64_kernel(const float *__restrict__ a, double *__restrict__ b, int64_t n)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = (double)a[i];
}

afn_status convert64to32(const double *a, float *b, int64_t count, cudaStream_t s)
{
    if (count <= 0) return AFN_OK;
    cvt64to32_kernel<<<(unsigned)((count + 255) / 256), 256, 0, s>>>(a, b, count);
    AFN_CUDA(cudaGetLastError());
    return AFN_OK;
}

afn_status convert32to64(const float *a, double *b, int64_t count, cudaStream_t s)
{
    if (count <= 0) return AFN_OK;
    cvt32to64_kernel<<<(unsigned)((count + 255) / 256), 256, 0, s>>>(a, b, count);
    AFN_CUDA(cudaGetLastError());
    return AFN_OK;
}

}  // namespace afn
