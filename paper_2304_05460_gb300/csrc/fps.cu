// fps.cu -- farthest point sampling (Alg. 6) and the landmark-first
// permutation (the 2x2 partition of Sec. 2).
//
// FPS runs one launch per step, so it never needs its whole grid resident at
// once and shares the GPU with other streams.  The distance-to-selected-set
// array d_j lives in global memory (L2-resident), points in SoA layout
// (coalesced).  A step = exact FP64 distance update against the last
// selected point (no FMA, dimensions in order), warp/block argmax with
// lowest-index ties, one partial per block; the last block to finish (an
// arrival counter) reduces the partials, writes the next selected index and
// marks it selected (d = -1).  The next launch reads that index, so the k-1
// launches are queued back to back without host round trips.
#include <algorithm>
#include <cfloat>
#include <climits>
#include <cmath>

#include "afn_device.cuh"
#include "afn_internal.cuh"

namespace afn {

static constexpr int FPS_T = 256;

__global__ void to_soa_kernel(const double *__restrict__ X, int64_t n, int d,
                              double *__restrict__ Xt)
{
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n * d) return;
    int64_t j = e / d;
    int t = (int)(e % d);
    Xt[(int64_t)t * n + j] = X[e];
}

// d_j = +inf (unvisited), -1 for the start point; idx[0] = start
__global__ void fps_init_kernel(int64_t n, int64_t start, double *__restrict__ dm,
                                int64_t *__restrict__ idx, unsigned int *cnt)
{
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j < n) dm[j] = (j == start) ? -1.0 : (double)INFINITY;
    if (j == 0) {
        idx[0] = start;
        *cnt = 0;
    }
}

__global__ void __launch_bounds__(FPS_T) fps_step_kernel(const double *__restrict__ Xt, int64_t n,
                                                         int d, int64_t it,
                                                         int64_t *__restrict__ idx,
                                                         double *__restrict__ dm,
                                                         double *partv, int64_t *parti,
                                                         unsigned int *cnt)
{
    __shared__ double xl[16];
    __shared__ double wv[FPS_T / 32];
    __shared__ int64_t wi[FPS_T / 32];
    __shared__ bool last;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t l = idx[it - 1];
    if (threadIdx.x < d) xl[threadIdx.x] = Xt[(int64_t)threadIdx.x * n + l];
    __syncthreads();
    double bv = -3.0;
    int64_t bi = LLONG_MAX;
    for (int64_t j = (int64_t)blockIdx.x * FPS_T + threadIdx.x; j < n;
         j += (int64_t)gridDim.x * FPS_T) {
        double v = dm[j];
        if (v >= 0.0) {
            double r2 = 0.0;
            for (int t = 0; t < d; ++t) {
                double u = __dsub_rn(Xt[(int64_t)t * n + j], xl[t]);
                r2 = __dadd_rn(r2, __dmul_rn(u, u));
            }
            if (r2 < v) {
                v = r2;
                dm[j] = v;
            }
        }
        if (better_max(v, j, bv, bi)) { bv = v; bi = j; }
    }
    warp_argmax(bv, bi);
    if (lane == 0) { wv[wid] = bv; wi[wid] = bi; }
    __syncthreads();
    if (wid == 0) {
        bv = (lane < FPS_T / 32) ? wv[lane] : -3.0;
        bi = (lane < FPS_T / 32) ? wi[lane] : LLONG_MAX;
        warp_argmax(bv, bi);
        if (lane == 0) {
            partv[blockIdx.x] = bv;
            parti[blockIdx.x] = bi;
            __threadfence();
            last = atomicAdd(cnt, 1u) == gridDim.x - 1;
        }
    }
    __syncthreads();
    if (!last) return;
    // the last block: every thread reads partials (one or two loads in flight
    // per thread rather than a serial chain in one warp), then the block argmax
    __threadfence();
    double v = -3.0;
    int64_t ii = LLONG_MAX;
    for (unsigned b = threadIdx.x; b < gridDim.x; b += FPS_T) {
        double v2 = __ldcg(partv + b);
        int64_t i2 = __ldcg(parti + b);
        if (better_max(v2, i2, v, ii)) { v = v2; ii = i2; }
    }
    warp_argmax(v, ii);
    __syncthreads();                       // wv / wi of the first reduction are read
    if (lane == 0) { wv[wid] = v; wi[wid] = ii; }
    __syncthreads();
    if (wid == 0) {
        v = (lane < FPS_T / 32) ? wv[lane] : -3.0;
        ii = (lane < FPS_T / 32) ? wi[lane] : LLONG_MAX;
        warp_argmax(v, ii);
        if (lane == 0) {
            idx[it] = ii;
            dm[ii] = -1.0;
            *cnt = 0;
        }
    }
}

afn_status fps_run(const double *X, int64_t n, int d, int64_t k, int64_t start, int64_t *idx,
                   int *status, cudaStream_t s)
{
    if (k <= 0) return AFN_OK;
    if (k > n || start < 0 || start >= n || d < 1 || d > 16) {
        set_error("fps: bad arguments (n=%lld d=%d k=%lld start=%lld)", (long long)n, d,
                  (long long)k, (long long)start);
        return AFN_ERR_ARG;
    }
    (void)status;
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    // one point per thread up to two blocks per SM: a step is a short chain of
    // FP64 operations per point (GB300 retires few FP64 operations per cycle), so
    // spreading the points over every SM shortens each of the k - 1 steps
    const int nb = (int)std::max<int64_t>(1, std::min<int64_t>((n + FPS_T - 1) / FPS_T,
                                                               (int64_t)sms * 2));
    DevBuf xt, dm, pv, pi, cnt;
    AFN_TRY(xt.alloc(sizeof(double) * (size_t)(n * d)));
    AFN_TRY(dm.alloc(sizeof(double) * (size_t)n));
    AFN_TRY(pv.alloc(sizeof(double) * nb));
    AFN_TRY(pi.alloc(sizeof(int64_t) * nb));
    AFN_TRY(cnt.alloc(sizeof(unsigned int)));
    const int64_t tot = n * d;
    to_soa_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(X, n, d, xt.as<double>());
    fps_init_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, start, dm.as<double>(), idx,
                                                                  cnt.as<unsigned int>());
    for (int64_t it = 1; it < k; ++it)
        fps_step_kernel<<<nb, FPS_T, 0, s>>>(xt.as<double>(), n, d, it, idx, dm.as<double>(),
                                             pv.as<double>(), pi.as<int64_t>(),
                                             cnt.as<unsigned int>());
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "fps launch");
    // the temporaries are released on stream s after the steps that use them
    return AFN_OK;
}

// ------------------------------------------------------- centroid start --
// Alg. 6's start: the point nearest the centroid.  Each coordinate of the
// centroid is summed over j = 0..n-1 in order by one thread, so the value is
// the same as a sequential loop; the argmin takes the lowest index on ties.
__global__ void centroid_kernel(const double *__restrict__ X, int64_t n, int d,
                                double *__restrict__ c)
{
    int t = threadIdx.x;
    if (t >= d) return;
    double s = 0.0;
    for (int64_t j = 0; j < n; ++j) s = __dadd_rn(s, X[j * d + t]);
    c[t] = s / (double)n;
}

__global__ void argmin_dist_kernel(const double *__restrict__ X, int64_t n, int d,
                                   const double *__restrict__ c, int64_t *out)
{
    __shared__ double wv[32];
    __shared__ int64_t wi[32];
    double bv = -DBL_MAX;   // maximise -r2 (lowest index ties)
    int64_t bi = LLONG_MAX;
    for (int64_t j = threadIdx.x; j < n; j += blockDim.x) {
        double r2 = sqdist_exact(X + j * d, c, d);
        if (better_max(-r2, j, bv, bi)) { bv = -r2; bi = j; }
    }
    warp_argmax(bv, bi);
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) { wv[wid] = bv; wi[wid] = bi; }
    __syncthreads();
    if (wid == 0) {
        int nw = blockDim.x / 32;
        bv = lane < nw ? wv[lane] : -DBL_MAX;
        bi = lane < nw ? wi[lane] : LLONG_MAX;
        warp_argmax(bv, bi);
        if (lane == 0) *out = bi;
    }
}

afn_status centroid_start(const double *X, int64_t n, int d, int64_t *out, cudaStream_t s)
{
    DevBuf c;
    AFN_TRY(c.alloc(sizeof(double) * 16));
    centroid_kernel<<<1, 32, 0, s>>>(X, n, d, c.as<double>());
    argmin_dist_kernel<<<1, 1024, 0, s>>>(X, n, d, c.as<double>(), out);
    AFN_CUDA(cudaGetLastError());
    AFN_CUDA(cudaStreamSynchronize(s));
    return AFN_OK;
}

// ---------------------------------------------------------- permutation --
// perm = [landmarks in selection order ; the others in ascending index].
__global__ void mark_kernel(const int64_t *__restrict__ lm, int64_t k, unsigned char *mark)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < k) mark[lm[i]] = 1;
}

__global__ void perm_kernel(const int64_t *__restrict__ lm, int64_t k, int64_t n,
                            const unsigned char *__restrict__ mark, int64_t *__restrict__ perm)
{
    // one block of 1024 threads; thread t scans a contiguous range
    __shared__ int64_t cnt[1024];
    const int t = threadIdx.x;
    const int64_t per = (n + 1023) / 1024;
    const int64_t a = min(n, t * per), b = min(n, a + per);
    int64_t c = 0;
    for (int64_t j = a; j < b; ++j) c += mark[j] ? 0 : 1;
    cnt[t] = c;
    __syncthreads();
    // inclusive scan (Hillis-Steele)
    for (int o = 1; o < 1024; o <<= 1) {
        int64_t v = (t >= o) ? cnt[t - o] : 0;
        __syncthreads();
        cnt[t] += v;
        __syncthreads();
    }
    int64_t pos = k + cnt[t] - c;
    for (int64_t j = a; j < b; ++j)
        if (!mark[j]) perm[pos++] = j;
    for (int64_t i = t; i < k; i += 1024) perm[i] = lm[i];
}

afn_status build_perm(const int64_t *landmarks, int64_t k, int64_t n, int64_t *perm,
                      cudaStream_t s)
{
    DevBuf mark;
    AFN_TRY(mark.alloc((size_t)n));
    AFN_CUDA(cudaMemsetAsync(mark.p, 0, (size_t)n, s));
    if (k > 0) mark_kernel<<<(unsigned)((k + 255) / 256), 256, 0, s>>>(landmarks, k, mark.as<unsigned char>());
    perm_kernel<<<1, 1024, 0, s>>>(landmarks, k, n, mark.as<unsigned char>(), perm);
    AFN_CUDA(cudaGetLastError());
    AFN_CUDA(cudaStreamSynchronize(s));
    return AFN_OK;
}

__global__ void gather_kernel(const double *__restrict__ X, const int64_t *__restrict__ perm,
                              int64_t n, int d, double *__restrict__ Xp)
{
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n * d) return;
    int64_t p = e / d;
    int t = (int)(e % d);
    Xp[e] = X[perm[p] * d + t];
}

afn_status gather_points(const double *X, const int64_t *perm, int64_t n, int d, double *Xp,
                         cudaStream_t s)
{
    int64_t tot = n * d;
    if (tot == 0) return AFN_OK;
    gather_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(X, perm, n, d, Xp);
    AFN_CUDA(cudaGetLastError());
    return AFN_OK;
}

}  // namespace afn
