// rank.cu -- Nystrom rank estimation, Alg. 4, on the device.
//
//   X_m  = m uniform draws (SplitMix64 partial Fisher-Yates, drawn on the
//          host as indices), coordinates scaled by (m/n)^(1/d);
//   o    = FPS order of X_m from index 0 (Alg. 6, fps.cu);
//   K_o  = K(X_m[o], X_m[o]);  theta = 0.1 ||K_o||_2;
//   E_r  = Schur complement of K_o after its first r pivots (Cholesky in
//          FPS order; a pivot <= m 2^-52 max diag is treated as zero);
//   r    = smallest rank with ||E_r||_2 < theta, by bisection over r (E_{r+1}
//          is a Schur complement of E_r, so its norm cannot grow);
//   k    = ceil(r n / m) if r n / m >= 2000, else the number of eigenvalues
//          of K(X_m, X_m) (unscaled points) above 0.1 mu; clipped to
//          [1, min(k_max, n)].
// Eigenvalue facts come from a Householder tridiagonalisation (one
// cooperative launch, two bounded grid barriers per column) and Sturm
// sequence counts on the tridiagonal.
#include <algorithm>
#include <cfloat>
#include <cmath>
#include <vector>

#include "afn_device.cuh"
#include "afn_internal.cuh"

namespace afn {

static constexpr int TT = 256;                              // threads per block
static constexpr uint64_t TRI_LIMIT_NS = 2000000000ull;     // 2 s per barrier wait
static constexpr int MMAX = 2048;

__device__ __forceinline__ double block_sum(double v, double *red)
{
    v = warp_sum(v);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double s = 0.0;
    for (int w = 0; w < TT / 32; ++w) s += red[w];
    __syncthreads();
    return s;
}

// Householder tridiagonalisation of the symmetric m x m row-major A (in
// place), Golub & Van Loan Alg. 8.3.1 restated: for column j, v from
// A[j+1:, j], beta = 2 / v^T v, p = beta A22 v, w = p - (beta/2)(p^T v) v,
// A22 -= v w^T + w v^T.  Rows of A22 are dealt round-robin to the blocks.
__global__ void __launch_bounds__(TT) tridiag_kernel(double *A, int m, double *dg, double *of,
                                                     double *pg, double *part,
                                                     unsigned int *bar, int *err)
{
    __shared__ double v[MMAX];
    __shared__ double w[MMAX];
    __shared__ double red[TT / 32];
    const unsigned nb = gridDim.x;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int j = 0; j + 2 < m; ++j) {
        const int len = m - j - 1;
        double loc = 0.0;
        for (int i = threadIdx.x; i < len; i += TT) {
            double x = __ldcg(A + (int64_t)(j + 1 + i) * m + j);
            v[i] = x;
            loc += x * x;
        }
        __syncthreads();
        const double nx = sqrt(block_sum(loc, red));
        const double x0 = v[0];
        const double ajj = __ldcg(A + (int64_t)j * m + j);
        if (nx == 0.0) {
            if (blockIdx.x == 0 && threadIdx.x == 0) { dg[j] = ajj; of[j] = 0.0; }
            continue;
        }
        const double alpha = (x0 >= 0.0) ? -nx : nx;
        __syncthreads();
        if (threadIdx.x == 0) v[0] = x0 - alpha;
        __syncthreads();
        loc = 0.0;
        for (int i = threadIdx.x; i < len; i += TT) loc += v[i] * v[i];
        const double vv = block_sum(loc, red);
        if (blockIdx.x == 0 && threadIdx.x == 0) { dg[j] = ajj; of[j] = alpha; }
        if (vv == 0.0) continue;
        const double beta = 2.0 / vv;
        // p = beta A22 v on this block's rows (warp per row)
        double pvl = 0.0;
        for (int a = blockIdx.x + nb * wid; a < len; a += nb * (TT / 32)) {
            const double *row = A + (int64_t)(j + 1 + a) * m + j + 1;
            double s = 0.0;
            for (int c = lane; c < len; c += 32) s += __ldcg(row + c) * v[c];
            s = warp_sum(s) * beta;
            if (lane == 0) {
                pg[a] = s;
                pvl += s * v[a];
            }
        }
        const double pvb = block_sum(lane == 0 ? pvl : 0.0, red);
        if (threadIdx.x == 0) part[blockIdx.x] = pvb;
        if (!grid_barrier(bar, bar + 1, nb, err, TRI_LIMIT_NS)) return;
        double pv = 0.0;
        for (unsigned b = 0; b < nb; ++b) pv += __ldcg(part + b);
        const double kk = 0.5 * beta * pv;
        for (int i = threadIdx.x; i < len; i += TT) w[i] = __ldcg(pg + i) - kk * v[i];
        __syncthreads();
        for (int a = blockIdx.x + nb * wid; a < len; a += nb * (TT / 32)) {
            double *row = A + (int64_t)(j + 1 + a) * m + j + 1;
            const double va = v[a], wa = w[a];
            for (int c = lane; c < len; c += 32) row[c] = __ldcg(row + c) - va * w[c] - wa * v[c];
        }
        if (!grid_barrier(bar, bar + 1, nb, err, TRI_LIMIT_NS)) return;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        if (m >= 2) {
            dg[m - 2] = __ldcg(A + (int64_t)(m - 2) * m + m - 2);
            of[m - 2] = __ldcg(A + (int64_t)(m - 1) * m + m - 2);
        }
        if (m >= 1) dg[m - 1] = __ldcg(A + (int64_t)(m - 1) * m + m - 1);
    }
}

// Sturm count: eigenvalues of the tridiagonal below sigma = factor * (*base)
__device__ int sturm_count_dev(const double *dg, const double *of, int m, double sigma)
{
    int cnt = 0;
    double q = 1.0;
    for (int i = 0; i < m; ++i) {
        double e2 = (i > 0) ? of[i - 1] * of[i - 1] : 0.0;
        q = (dg[i] - sigma) - (i > 0 ? e2 / q : 0.0);
        if (q == 0.0) q = -1e-300;
        if (q < 0.0) ++cnt;
    }
    return cnt;
}

__global__ void sturm_kernel(const double *dg, const double *of, int m, const double *base,
                             double factor, int *out)
{
    double sigma = base ? factor * (*base) : factor;
    *out = sturm_count_dev(dg, of, m, sigma);
}

// largest eigenvalue by bisection on the Sturm count (Gershgorin start).
// The bisection takes the same midpoints as a sequential loop, eight levels
// at a time: thread t of the 255 evaluates the Sturm count at node t of the
// next eight levels' subtree (its interval reached from [lo, hi] by the same
// midpoint arithmetic), and thread 0 then walks the subtree.
__global__ void __launch_bounds__(256) lmax_kernel(const double *dg, const double *of, int m, double *out)
{
    __shared__ double slo, shi;
    __shared__ int done;
    __shared__ unsigned char top[256];   // count == m at node t (mid is above every eigenvalue)
    if (threadIdx.x == 0) {
        double lo = DBL_MAX, hi = -DBL_MAX;
        for (int i = 0; i < m; ++i) {
            double rad = (i > 0 ? fabs(of[i - 1]) : 0.0) + (i + 1 < m ? fabs(of[i]) : 0.0);
            lo = fmin(lo, dg[i] - rad);
            hi = fmax(hi, dg[i] + rad);
        }
        slo = lo;
        shi = hi;
        done = 0;
    }
    __syncthreads();
    for (int round = 0; round < 25 && !done; ++round) {
        const int t = threadIdx.x;      // node t in 1..255 (BFS order, root 1)
        if (t >= 1) {
            // the path from the root: bits of t below its leading one, high to low
            int depth = 31 - __clz(t);
            double lo = slo, hi = shi;
            bool ok = true;
            for (int b = depth - 1; b >= 0; --b) {
                const double mid = 0.5 * (lo + hi);
                if (!(mid > lo && mid < hi)) { ok = false; break; }
                if ((t >> b) & 1) lo = mid; else hi = mid;
            }
            const double mid = 0.5 * (lo + hi);
            top[t] = (ok && mid > lo && mid < hi && sturm_count_dev(dg, of, m, mid) == m) ? 1 : 0;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            double lo = slo, hi = shi;
            int node = 1;
            for (int lev = 0; lev < 8; ++lev) {
                const double mid = 0.5 * (lo + hi);
                if (!(mid > lo && mid < hi)) { done = 1; break; }
                if (top[node]) { hi = mid; node = 2 * node; } else { lo = mid; node = 2 * node + 1; }
            }
            slo = lo;
            shi = hi;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = 0.5 * (slo + shi);
}

// A <- factor * (*base) I - A  (sz x sz)
__global__ void shift_neg_kernel(double *A, int sz, const double *base, double factor)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)sz * sz) return;
    const int64_t i = e / sz, j = e % sz;
    A[e] = (i == j ? factor * (*base) : 0.0) - A[e];
}

__global__ void gather_scale_kernel(const double *__restrict__ X, const int64_t *__restrict__ idx,
                                    int64_t m, int d, double sc, double *__restrict__ out)
{
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= m * d) return;
    int64_t i = e / d;
    int t = (int)(e % d);
    out[e] = (sc == 1.0) ? X[idx[i] * d + t] : X[idx[i] * d + t] * sc;
}

// E[a, b] = Ko[r+a, r+b] - sum_{t<r} Lo[r+a, t] Lo[r+b, t]  (s = m - r)
__global__ void __launch_bounds__(256) schur_kernel(const double *__restrict__ Ko,
                                                    const double *__restrict__ Lo, int m, int r,
                                                    double *__restrict__ E)
{
    const int s = m - r;
    const int r0 = blockIdx.y * 64, c0 = blockIdx.x * 64;
    __shared__ double pa[32][65];
    __shared__ double pb[32][65];
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    double acc[4][4] = {};
    for (int t0 = 0; t0 < r; t0 += 32) {
        __syncthreads();
        for (int e = threadIdx.x; e < 64 * 32; e += 256) {
            int q = e / 32, t = e % 32;
            int ga = r0 + q, gb = c0 + q, gt = t0 + t;
            pa[t][q] = (ga < s && gt < r) ? Lo[(int64_t)(r + ga) * m + gt] : 0.0;
            pb[t][q] = (gb < s && gt < r) ? Lo[(int64_t)(r + gb) * m + gt] : 0.0;
        }
        __syncthreads();
        for (int t = 0; t < 32; ++t) {
            double a[4], b[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) { a[q] = pa[t][ty * 4 + q]; b[q] = pb[t][tx * 4 + q]; }
#pragma unroll
            for (int x = 0; x < 4; ++x)
#pragma unroll
                for (int y = 0; y < 4; ++y) acc[x][y] += a[x] * b[y];
        }
    }
#pragma unroll
    for (int x = 0; x < 4; ++x) {
        int ga = r0 + ty * 4 + x;
        if (ga >= s) continue;
#pragma unroll
        for (int y = 0; y < 4; ++y) {
            int gb = c0 + tx * 4 + y;
            if (gb < s) E[(int64_t)ga * s + gb] = Ko[(int64_t)(r + ga) * m + r + gb] - acc[x][y];
        }
    }
}

// tridiagonalise the s x s matrix in A (destroyed), results in dg/of
static afn_status tridiagonalize(double *A, int s, double *dg, double *of, int *err,
                                 cudaStream_t st)
{
    if (s <= 0) return AFN_OK;
    if (s > MMAX) {
        set_error("rank estimate: subsample size %d above %d", s, MMAX);
        return AFN_ERR_ARG;
    }
    int dev = 0, sms = 1, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, tridiag_kernel, TT, 0);
    int nb = std::max(1, std::min(std::min(sms * std::max(per, 1), sms), (s + 7) / 8));
    DevBuf pg, part, bar;
    AFN_TRY(pg.alloc(sizeof(double) * s));
    AFN_TRY(part.alloc(sizeof(double) * nb));
    AFN_TRY(bar.alloc(sizeof(unsigned int) * 2));
    AFN_CUDA(cudaMemsetAsync(bar.p, 0, sizeof(unsigned int) * 2, st));
    double *pgp = pg.as<double>(), *pp = part.as<double>();
    unsigned int *bp = bar.as<unsigned int>();
    void *args[] = {(void *)&A, (void *)&s, (void *)&dg, (void *)&of, (void *)&pgp, (void *)&pp,
                    (void *)&bp, (void *)&err};
    AFN_CUDA(cudaLaunchCooperativeKernel((void *)tridiag_kernel, dim3(nb), dim3(TT), args, 0, st));
    int he = 0;
    AFN_CUDA(cudaMemcpyAsync(&he, err, sizeof(int), cudaMemcpyDeviceToHost, st));
    AFN_CUDA(cudaStreamSynchronize(st));
    if (he == DEV_TIMEOUT) {
        set_error("tridiagonalisation: grid barrier wait exceeded its limit");
        return AFN_ERR_TIMEOUT;
    }
    return AFN_OK;
}

afn_status rank_estimate(const double *X, int64_t n, int d, KParams kp, int m, uint64_t seed,
                         int64_t k_max, int64_t *k_out, int64_t *r_out, int *branch_out, int *status,
                         cudaStream_t s)
{
    if (m > n) m = (int)n;
    if (m < 1) m = 1;
    if (m > MMAX) {
        set_error("rank estimate: m=%d above %d", m, MMAX);
        return AFN_ERR_ARG;
    }
    std::vector<int64_t> sub;
    uniform_sample_host(n, m, seed, sub);
    const double sc = pow((double)m / (double)n, 1.0 / (double)d);
    DevBuf dsub, Xs, o, Xo, Ko, T, Lo, E, dg, of, lm, cnt;
    AFN_TRY(dsub.alloc(sizeof(int64_t) * m));
    AFN_CUDA(cudaMemcpyAsync(dsub.p, sub.data(), sizeof(int64_t) * m, cudaMemcpyHostToDevice, s));
    AFN_TRY(Xs.alloc(sizeof(double) * m * d));
    unsigned g = (unsigned)(((int64_t)m * d + 255) / 256);
    gather_scale_kernel<<<g, 256, 0, s>>>(X, dsub.as<int64_t>(), m, d, sc, Xs.as<double>());
    AFN_TRY(o.alloc(sizeof(int64_t) * m));
    AFN_TRY(fps_run(Xs.as<double>(), m, d, m, 0, o.as<int64_t>(), status, s));
    AFN_TRY(Xo.alloc(sizeof(double) * m * d));
    gather_scale_kernel<<<g, 256, 0, s>>>(Xs.as<double>(), o.as<int64_t>(), m, d, 1.0, Xo.as<double>());
    const size_t mm = (size_t)m * m;
    AFN_TRY(Ko.alloc(sizeof(double) * mm));
    AFN_TRY(T.alloc(sizeof(double) * mm));
    AFN_TRY(Lo.alloc(sizeof(double) * mm));
    AFN_TRY(E.alloc(sizeof(double) * mm));
    AFN_TRY(dg.alloc(sizeof(double) * m));
    AFN_TRY(of.alloc(sizeof(double) * std::max(m, 2)));
    AFN_TRY(lm.alloc(sizeof(double)));
    AFN_TRY(cnt.alloc(sizeof(int)));
    AFN_TRY(kernel_block(Xo.as<double>(), m, Xo.as<double>(), m, d, kp, 0.0, Ko.as<double>(), m, s));
    // ||K_o||_2
    AFN_CUDA(cudaMemcpyAsync(T.p, Ko.p, sizeof(double) * mm, cudaMemcpyDeviceToDevice, s));
    AFN_CUDA(cudaMemsetAsync(status, 0, sizeof(int), s));
    AFN_TRY(tridiagonalize(T.as<double>(), m, dg.as<double>(), of.as<double>(), status, s));
    lmax_kernel<<<1, 256, 0, s>>>(dg.as<double>(), of.as<double>(), m, lm.as<double>());
    // Cholesky of K_o in FPS order with negligible pivots dropped
    AFN_CUDA(cudaMemcpyAsync(Lo.p, Ko.p, sizeof(double) * mm, cudaMemcpyDeviceToDevice, s));
    const double tiny = (double)m * 2.220446049250313e-16;   // max diag of K_o is 1
    AFN_TRY(cholesky64(Lo.as<double>(), m, status, s, tiny));
    // ||E_r||_2 < 0.1 ||K_o||_2  <=>  every eigenvalue of the Schur complement
    // E_r is below theta = 0.1 lambda_max(K_o)  <=>  theta I - E_r is positive
    // definite, which a Cholesky decides (a quarter of the flops of the
    // tridiagonalisation that the eigenvalue count would need)
    auto below = [&](int r, bool *res) -> afn_status {
        int sz = m - r;
        if (sz <= 0) { *res = true; return AFN_OK; }
        dim3 gg((unsigned)((sz + 63) / 64), (unsigned)((sz + 63) / 64));
        schur_kernel<<<gg, 256, 0, s>>>(Ko.as<double>(), Lo.as<double>(), m, r, E.as<double>());
        const int64_t tot = (int64_t)sz * sz;
        shift_neg_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(E.as<double>(), sz,
                                                                       lm.as<double>(), 0.1);
        AFN_TRY(cholesky64(E.as<double>(), sz, status, s, -1.0));
        int hs = 0;
        AFN_CUDA(cudaMemcpyAsync(&hs, status, sizeof(int), cudaMemcpyDeviceToHost, s));
        AFN_CUDA(cudaStreamSynchronize(s));
        *res = (hs == 0);
        return AFN_OK;
    };
    int lo = 1, hi = m;
    while (lo < hi) {
        int mid = lo + (hi - lo) / 2;
        bool b = false;
        AFN_TRY(below(mid, &b));
        if (b) hi = mid; else lo = mid + 1;
    }
    const int64_t r = lo;
    int64_t k;
    int branch;
    if (r * n >= 2000 * (int64_t)m) {
        k = (r * n + m - 1) / m;
        branch = 0;
    } else {
        gather_scale_kernel<<<g, 256, 0, s>>>(X, dsub.as<int64_t>(), m, d, 1.0, Xs.as<double>());
        AFN_TRY(kernel_block(Xs.as<double>(), m, Xs.as<double>(), m, d, kp, 0.0, T.as<double>(), m, s));
        AFN_CUDA(cudaMemsetAsync(status, 0, sizeof(int), s));
        AFN_TRY(tridiagonalize(T.as<double>(), m, dg.as<double>(), of.as<double>(), status, s));
        sturm_kernel<<<1, 1, 0, s>>>(dg.as<double>(), of.as<double>(), m, nullptr, 0.1 * kp.mu,
                                     cnt.as<int>());
        int hc = 0;
        AFN_CUDA(cudaMemcpyAsync(&hc, cnt.p, sizeof(int), cudaMemcpyDeviceToHost, s));
        AFN_CUDA(cudaStreamSynchronize(s));
        k = m - hc;
        branch = 1;
    }
    int64_t cap = std::min<int64_t>(k_max, n);
    k = std::max<int64_t>(1, std::min<int64_t>(k, cap));
    *k_out = k;
    if (r_out) *r_out = r;
    if (branch_out) *branch_out = branch;
    AFN_CUDA(cudaGetLastError());
    return AFN_OK;
}

}  // namespace afn
