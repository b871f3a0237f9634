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
    matvec32_kernel<D, NR, KER><<<grid, NT, 0, s>>>(Xs, n, P, n, part, chunk);
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
        int b = piece(nrhs - c0, 32);
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
    return sizeof(double) * (size_t)pick_js(n) * (size_t)std::min(std::max(nrhs, 1), 8) *
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
    default: matvec64_kernel<D, 8><<<grid, NT, 0, s>>>(X, d, n, kernel, l, P, n, part, chunk); break;
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
        int b = piece(nrhs - c0, 8);
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
