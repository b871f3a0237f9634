// fps.cu -- farthest point sampling (Alg. 6) and the landmark-first
// permutation (the 2x2 partition of Sec. 2).
//
// FPS is one persistent cooperative launch.  Each thread owns up to PPT
// points (j = gtid + s*T) and keeps their distance-to-selected-set entries in
// registers for all k-1 steps; points are read in SoA layout (coalesced) from
// L2.  One step = exact FP64 distance update (no FMA, dimensions in order),
// warp/block argmax with lowest-index ties, one partial per block, one grid
// barrier (bounded wait), and a redundant in-order reduction of the partials
// by every block.  Partials are double-buffered by step parity, so one
// barrier per step suffices.
#include <algorithm>
#include <cfloat>
#include <climits>
#include <cmath>

#include "afn_device.cuh"
#include "afn_internal.cuh"

namespace afn {

static constexpr int FPS_T = 256;
static constexpr uint64_t BARRIER_LIMIT_NS = 2000000000ull;   // 2 s per wait

__global__ void to_soa_kernel(const double *__restrict__ X, int64_t n, int d,
                              double *__restrict__ Xt)
{
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n * d) return;
    int64_t j = e / d;
    int t = (int)(e % d);
    Xt[(int64_t)t * n + j] = X[e];
}

template <int PPT>
__global__ void __launch_bounds__(FPS_T) fps_kernel(const double *__restrict__ Xt, int64_t n,
                                                    int d, int64_t k, int64_t start,
                                                    int64_t *__restrict__ idx,
                                                    double *partv, int64_t *parti,
                                                    unsigned int *bar, int *err)
{
    __shared__ double xl[16];
    __shared__ double wv[FPS_T / 32];
    __shared__ int64_t wi[FPS_T / 32];
    __shared__ int64_t lsel;
    const int64_t T = (int64_t)gridDim.x * FPS_T;
    const int64_t gtid = (int64_t)blockIdx.x * FPS_T + threadIdx.x;
    const unsigned nb = gridDim.x;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;

    double dm[PPT];
#pragma unroll
    for (int s = 0; s < PPT; ++s) {
        int64_t j = gtid + s * T;
        dm[s] = (j < n) ? ((j == start) ? -1.0 : (double)INFINITY) : -2.0;   // unvisited, selected, absent
    }
    if (gtid == 0) idx[0] = start;
    int64_t l = start;
    for (int64_t it = 1; it < k; ++it) {
        if (threadIdx.x < d) xl[threadIdx.x] = Xt[(int64_t)threadIdx.x * n + l];
        __syncthreads();
        double bv = -3.0;
        int64_t bi = LLONG_MAX;
#pragma unroll
        for (int s = 0; s < PPT; ++s) {
            int64_t j = gtid + s * T;
            if (dm[s] >= 0.0) {
                double r2 = 0.0;
                for (int t = 0; t < d; ++t) {
                    double u = __dsub_rn(Xt[(int64_t)t * n + j], xl[t]);
                    r2 = __dadd_rn(r2, __dmul_rn(u, u));
                }
                if (r2 < dm[s]) dm[s] = r2;
            }
            if (better_max(dm[s], j, bv, bi)) { bv = dm[s]; bi = j; }
        }
        warp_argmax(bv, bi);
        if (lane == 0) { wv[wid] = bv; wi[wid] = bi; }
        __syncthreads();
        if (wid == 0) {
            bv = (lane < FPS_T / 32) ? wv[lane] : -3.0;
            bi = (lane < FPS_T / 32) ? wi[lane] : LLONG_MAX;
            warp_argmax(bv, bi);
            if (lane == 0) {
                partv[(it & 1) * nb + blockIdx.x] = bv;
                parti[(it & 1) * nb + blockIdx.x] = bi;
            }
        }
        if (!grid_barrier(bar, bar + 1, nb, err, BARRIER_LIMIT_NS)) return;
        if (wid == 0) {
            double v = -3.0;
            int64_t ii = LLONG_MAX;
            for (unsigned b = lane; b < nb; b += 32) {
                double v2 = __ldcg(partv + (it & 1) * nb + b);
                int64_t i2 = __ldcg(parti + (it & 1) * nb + b);
                if (better_max(v2, i2, v, ii)) { v = v2; ii = i2; }
            }
            warp_argmax(v, ii);
            if (lane == 0) lsel = ii;
        }
        __syncthreads();
        l = lsel;
        if (gtid == 0) idx[it] = l;
#pragma unroll
        for (int s = 0; s < PPT; ++s)
            if (gtid + s * T == l) dm[s] = -1.0;
    }
}

template <int PPT>
static cudaError_t launch_fps(int nb, const double *Xt, int64_t n, int d, int64_t k,
                              int64_t start, int64_t *idx, double *pv, int64_t *pi,
                              unsigned int *bar, int *err, cudaStream_t s)
{
    void *args[] = {(void *)&Xt, (void *)&n, (void *)&d, (void *)&k, (void *)&start,
                    (void *)&idx, (void *)&pv, (void *)&pi, (void *)&bar, (void *)&err};
    return cudaLaunchCooperativeKernel((void *)fps_kernel<PPT>, dim3(nb), dim3(FPS_T), args, 0, s);
}

template <int PPT>
static int max_coop_blocks()
{
    int dev = 0, sms = 1, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fps_kernel<PPT>, FPS_T, 0);
    return std::max(1, per) * sms;
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
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int nb = (int)std::min<int64_t>((n + 2 * FPS_T - 1) / (2 * FPS_T), sms);
    nb = std::max(nb, 1);
    int64_t T = (int64_t)nb * FPS_T;
    int64_t ppt = (n + T - 1) / T;
    int P = ppt <= 1 ? 1 : ppt <= 2 ? 2 : ppt <= 4 ? 4 : ppt <= 8 ? 8 : ppt <= 16 ? 16 : 32;
    if (ppt > 32) {
        set_error("fps: n=%lld too large for one cooperative launch", (long long)n);
        return AFN_ERR_ARG;
    }
    int cap = 0;
    switch (P) {
    case 1: cap = max_coop_blocks<1>(); break;
    case 2: cap = max_coop_blocks<2>(); break;
    case 4: cap = max_coop_blocks<4>(); break;
    case 8: cap = max_coop_blocks<8>(); break;
    case 16: cap = max_coop_blocks<16>(); break;
    default: cap = max_coop_blocks<32>(); break;
    }
    if (nb > cap) {
        set_error("fps: %d blocks exceed the co-resident limit %d", nb, cap);
        return AFN_ERR_ARG;
    }
    DevBuf xt, pv, pi, bar;
    AFN_TRY(xt.alloc(sizeof(double) * (size_t)(n * d)));
    AFN_TRY(pv.alloc(sizeof(double) * 2 * nb));
    AFN_TRY(pi.alloc(sizeof(int64_t) * 2 * nb));
    AFN_TRY(bar.alloc(sizeof(unsigned int) * 2));
    AFN_CUDA(cudaMemsetAsync(bar.p, 0, sizeof(unsigned int) * 2, s));
    AFN_CUDA(cudaMemsetAsync(status, 0, sizeof(int), s));
    int64_t tot = n * d;
    to_soa_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(X, n, d, xt.as<double>());
    cudaError_t e;
    switch (P) {
    case 1: e = launch_fps<1>(nb, xt.as<double>(), n, d, k, start, idx, pv.as<double>(), pi.as<int64_t>(), bar.as<unsigned int>(), status, s); break;
    case 2: e = launch_fps<2>(nb, xt.as<double>(), n, d, k, start, idx, pv.as<double>(), pi.as<int64_t>(), bar.as<unsigned int>(), status, s); break;
    case 4: e = launch_fps<4>(nb, xt.as<double>(), n, d, k, start, idx, pv.as<double>(), pi.as<int64_t>(), bar.as<unsigned int>(), status, s); break;
    case 8: e = launch_fps<8>(nb, xt.as<double>(), n, d, k, start, idx, pv.as<double>(), pi.as<int64_t>(), bar.as<unsigned int>(), status, s); break;
    case 16: e = launch_fps<16>(nb, xt.as<double>(), n, d, k, start, idx, pv.as<double>(), pi.as<int64_t>(), bar.as<unsigned int>(), status, s); break;
    default: e = launch_fps<32>(nb, xt.as<double>(), n, d, k, start, idx, pv.as<double>(), pi.as<int64_t>(), bar.as<unsigned int>(), status, s); break;
    }
    if (e != cudaSuccess) return cuda_fail(e, "fps cooperative launch");
    // the temporaries are released at scope exit: make sure the kernel is done
    AFN_CUDA(cudaStreamSynchronize(s));
    int hs = 0;
    AFN_CUDA(cudaMemcpyAsync(&hs, status, sizeof(int), cudaMemcpyDeviceToHost, s));
    AFN_CUDA(cudaStreamSynchronize(s));
    if (hs == DEV_TIMEOUT) {
        set_error("fps: grid barrier wait exceeded its limit");
        return AFN_ERR_TIMEOUT;
    }
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
