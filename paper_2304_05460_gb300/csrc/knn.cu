// knn.cu -- FSAI sparsity pattern (Sec. 3.1): row i of the Schur rows holds
// its w-1 nearest lower-numbered points, ordered by (FP64 squared distance,
// index), then i itself.
//
// One thread per row; a CTA of 128 consecutive rows streams the points
// j < (its last row) through shared memory tiles and every lane reads the
// same x_j (broadcast).  The selection uses exact FP64 distances (no FMA,
// dimensions in order), so it is identical to a sequential scan.  Each
// thread keeps its candidates in a max-heap ordered by (distance, index),
// the distances compared through the integer order of their bits (no FP64
// compares: this GPU's FP64 rate is a small fraction of its FP32 rate); a new
// j replaces the root only when strictly closer (j grows, so an equal
// distance never wins).  Once the list is full, a j is first tested in
// FP32: with every coordinate of magnitude <= M, the FP32 squared distance
// z of a pair whose exact one is r2 satisfies |z - r2| <=
// z <= (1 + gamma) (r2 + delta (2 sqrt(d r2) + d delta)) with delta about
// 2^-22 M (the rounded coordinates and their rounded difference) and gamma <
// (d + 2) 2^-24 (d + 1 roundings of the squares and the running sum), so a j
// whose z exceeds that bound at r2 = wv cannot be strictly closer and is
// skipped without computing its FP64 distance.  The bound is evaluated in
// FP32 with upward rounding throughout, so it never falls below the real
// bound.  The heaviest CTAs (largest i) start first.
#include <algorithm>
#include <cfloat>
#include <cmath>

#include "afn_device.cuh"
#include "afn_internal.cuh"

namespace afn {

static constexpr int KR = 128;    // rows per CTA
static constexpr int KTJ = 128;   // points per tile

// largest |coordinate| (as the bits of a non-negative double, whose integer
// order is its numeric order)
__global__ void maxabs_kernel(const double *__restrict__ X, int64_t count,
                              unsigned long long *__restrict__ out)
{
    double m = 0.0;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < count;
         e += (int64_t)gridDim.x * blockDim.x)
        m = fmax(m, fabs(X[e]));
    m = warp_max_d(m);
    if ((threadIdx.x & 31) == 0) atomicMax(out, (unsigned long long)__double_as_longlong(m));
}

// (key, j) order of the candidate list: the bits of a non-negative double
// compare as integers in its numeric order; ties go to the larger index.
__device__ __forceinline__ bool knn_after(unsigned long long ka, int32_t ja, unsigned long long kb,
                                          int32_t jb)
{
    return ka > kb || (ka == kb && ja > jb);
}

// put (key, j) at slot p of the max-heap hk/hj of size cnt and sift it down
template <int CAP>
__device__ __forceinline__ void knn_sift(unsigned long long (&hk)[CAP], int32_t (&hj)[CAP], int cnt,
                                         int p, unsigned long long key, int32_t j)
{
    for (;;) {
        int c = 2 * p + 1;
        if (c >= cnt) break;
        if (c + 1 < cnt && knn_after(hk[c + 1], hj[c + 1], hk[c], hj[c])) ++c;
        if (!knn_after(hk[c], hj[c], key, j)) break;
        hk[p] = hk[c];
        hj[p] = hj[c];
        p = c;
    }
    hk[p] = key;
    hj[p] = j;
}

template <int CAP>
__global__ void __launch_bounds__(KR) knn_kernel(const double *__restrict__ X, int64_t nr, int d,
                                                 int w, const unsigned long long *__restrict__ maxabs,
                                                 int32_t *__restrict__ pat)
{
    __shared__ double xs[KTJ * 16];
    __shared__ float xf[KTJ * 16];
    const int64_t rb = (int64_t)gridDim.x - 1 - blockIdx.x;   // heavy blocks first
    const int64_t i = rb * KR + threadIdx.x;
    const int64_t ilast = min(nr - 1, rb * KR + KR - 1);
    // error bound of the FP32 pre-test (see the file comment), rounded so
    // that the FP32 evaluation below is an upper bound of the real one
    const double M = __longlong_as_double((long long)*maxabs);
    const float dlt = __double2float_ru(M * 0x1p-22 * (1.0 + 0x1p-20));
    const float den = __double2float_rd(1.0 - (d + 2) * 0x1p-24);
    const float fd = (float)d;
    const float ddl = __fmul_ru(fd, dlt);
    double xi[16];
    float xif[16];
    for (int t = 0; t < d; ++t) {
        xi[t] = (i < nr) ? X[i * d + t] : 0.0;
        xif[t] = (float)xi[t];
    }
    // candidates: a max-heap on (distance bits, index) once full
    unsigned long long hk[CAP];
    int32_t hj[CAP];
    const int m = (i < nr) ? (int)min(i, (int64_t)(w - 1)) : 0;
    int cnt = 0;
    float zcut = INFINITY;          // skip j when its FP32 distance exceeds this
    for (int64_t jt = 0; jt < ilast; jt += KTJ) {
        __syncthreads();
        for (int e = threadIdx.x; e < KTJ * d; e += KR) {
            int64_t j = jt + e / d;
            const double v = (j < nr) ? X[jt * d + e] : 0.0;
            xs[e] = v;
            xf[e] = (float)v;
        }
        __syncthreads();
        const int64_t jend = min((int64_t)KTJ, i - jt);   // only j < i
        for (int jj = 0; jj < jend && m > 0; ++jj) {
            if (cnt == m) {
                float z = 0.f;
                for (int t = 0; t < d; ++t) {
                    const float u = __fsub_rn(xif[t], xf[jj * d + t]);
                    z = __fadd_rn(z, __fmul_rn(u, u));
                }
                if (z > zcut) continue;
            }
            double r2 = 0.0;
            for (int t = 0; t < d; ++t) {
                double u = __dsub_rn(xi[t], xs[jj * d + t]);
                r2 = __dadd_rn(r2, __dmul_rn(u, u));
            }
            const unsigned long long key = (unsigned long long)__double_as_longlong(r2);
            const int32_t j = (int32_t)(jt + jj);
            bool changed = false;
            if (cnt < m) {
                hk[cnt] = key;
                hj[cnt] = j;
                if (++cnt == m) {
                    for (int p = cnt / 2 - 1; p >= 0; --p) knn_sift(hk, hj, cnt, p, hk[p], hj[p]);
                    changed = true;
                }
            } else if (key < hk[0]) {   // strictly closer: an equal distance never wins
                knn_sift(hk, hj, cnt, 0, key, j);
                changed = true;
            }
            if (changed) {
                // z > wv + bound(wv) implies r2 > wv, wv the worst candidate
                const float wv = __double2float_ru(__longlong_as_double((long long)hk[0]));
                const float sq = __fsqrt_ru(__fmul_ru(fd, wv));
                const float b = __fmul_ru(dlt, __fadd_ru(__fmul_ru(2.f, sq), ddl));
                zcut = __fdiv_ru(__fadd_ru(wv, b), den);
            }
        }
    }
    if (i >= nr) return;
    // heap sort: ascending (distance, index)
    for (int e = cnt - 1; e > 0; --e) {
        const unsigned long long k = hk[e];
        const int32_t jv = hj[e];
        hk[e] = hk[0];
        hj[e] = hj[0];
        knn_sift(hk, hj, e, 0, k, jv);
    }
    int32_t *row = pat + i * w;
    for (int p = 0; p < cnt; ++p) row[p] = hj[p];
    row[cnt] = (int32_t)i;
    for (int p = cnt + 1; p < w; ++p) row[p] = -1;
}

afn_status knn_pattern(const double *Xr, int64_t nr, int d, int w, int32_t *pat, cudaStream_t s)
{
    if (nr <= 0) return AFN_OK;
    if (d < 1 || d > 16 || w < 1 || w > 256) {
        set_error("knn: unsupported d=%d or w=%d (1<=d<=16, 1<=w<=256)", d, w);
        return AFN_ERR_ARG;
    }
    DevBuf mx;
    AFN_TRY(mx.alloc(sizeof(unsigned long long)));
    AFN_CUDA(cudaMemsetAsync(mx.p, 0, sizeof(unsigned long long), s));
    const int64_t cnt = nr * d;
    maxabs_kernel<<<(unsigned)std::min<int64_t>((cnt + 255) / 256, 1024), 256, 0, s>>>(
        Xr, cnt, mx.as<unsigned long long>());
    const unsigned long long *M = mx.as<unsigned long long>();
    unsigned grid = (unsigned)((nr + KR - 1) / KR);
    if (w <= 32) knn_kernel<31><<<grid, KR, 0, s>>>(Xr, nr, d, w, M, pat);
    else if (w <= 64) knn_kernel<63><<<grid, KR, 0, s>>>(Xr, nr, d, w, M, pat);
    else if (w <= 128) knn_kernel<127><<<grid, KR, 0, s>>>(Xr, nr, d, w, M, pat);
    else knn_kernel<255><<<grid, KR, 0, s>>>(Xr, nr, d, w, M, pat);
    AFN_CUDA(cudaGetLastError());
    // mx is released on stream s after the kernels that read it
    return AFN_OK;
}

}  // namespace afn
