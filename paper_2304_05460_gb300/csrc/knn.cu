// knn.cu -- FSAI sparsity pattern (Sec. 3.1): row i of the Schur rows holds
// its w-1 nearest lower-numbered points, ordered by (FP64 squared distance,
// index), then i itself.
//
// One thread per row; a CTA of 128 consecutive rows streams the points
// j < (its last row) through shared memory tiles and every lane reads the
// same x_j (broadcast).  Distances are exact FP64 (no FMA, dimensions in
// order), so the selection is identical to a sequential scan.  Each thread
// keeps an unsorted candidate list in local memory and the position of its
// worst entry; a new j replaces the worst only when strictly closer (j grows,
// so an equal distance never wins).  The heaviest CTAs (largest i) start
// first.
#include <algorithm>
#include <cfloat>
#include <cmath>

#include "afn_device.cuh"
#include "afn_internal.cuh"

namespace afn {

static constexpr int KR = 128;    // rows per CTA
static constexpr int KTJ = 128;   // points per tile

template <int CAP>
__global__ void __launch_bounds__(KR) knn_kernel(const double *__restrict__ X, int64_t nr, int d,
                                                 int w, int32_t *__restrict__ pat)
{
    __shared__ double xs[KTJ * 16];
    const int64_t rb = (int64_t)gridDim.x - 1 - blockIdx.x;   // heavy blocks first
    const int64_t i = rb * KR + threadIdx.x;
    const int64_t ilast = min(nr - 1, rb * KR + KR - 1);
    double xi[16];
    for (int t = 0; t < d; ++t) xi[t] = (i < nr) ? X[i * d + t] : 0.0;
    double bd[CAP];
    int32_t bj[CAP];
    const int64_t m = (i < nr) ? min(i, (int64_t)(w - 1)) : 0;
    int cnt = 0, worst = 0;
    double wv = (double)INFINITY;
    for (int64_t jt = 0; jt < ilast; jt += KTJ) {
        __syncthreads();
        for (int e = threadIdx.x; e < KTJ * d; e += KR) {
            int64_t j = jt + e / d;
            xs[e] = (j < nr) ? X[jt * d + e] : 0.0;
        }
        __syncthreads();
        const int64_t jend = min((int64_t)KTJ, i - jt);   // only j < i
        for (int jj = 0; jj < jend && m > 0; ++jj) {
            double r2 = 0.0;
            for (int t = 0; t < d; ++t) {
                double u = __dsub_rn(xi[t], xs[jj * d + t]);
                r2 = __dadd_rn(r2, __dmul_rn(u, u));
            }
            if (cnt < m) {
                bd[cnt] = r2;
                bj[cnt] = (int32_t)(jt + jj);
                ++cnt;
                if (cnt == m) {
                    worst = 0;
                    for (int q = 1; q < cnt; ++q)
                        if (bd[q] > bd[worst] || (bd[q] == bd[worst] && bj[q] > bj[worst])) worst = q;
                    wv = bd[worst];
                }
            } else if (r2 < wv) {
                bd[worst] = r2;
                bj[worst] = (int32_t)(jt + jj);
                worst = 0;
                for (int q = 1; q < cnt; ++q)
                    if (bd[q] > bd[worst] || (bd[q] == bd[worst] && bj[q] > bj[worst])) worst = q;
                wv = bd[worst];
            }
        }
    }
    if (i >= nr) return;
    // sort by (r2, j) ascending
    for (int a = 1; a < cnt; ++a) {
        double v = bd[a];
        int32_t jv = bj[a];
        int b = a - 1;
        while (b >= 0 && (bd[b] > v || (bd[b] == v && bj[b] > jv))) {
            bd[b + 1] = bd[b];
            bj[b + 1] = bj[b];
            --b;
        }
        bd[b + 1] = v;
        bj[b + 1] = jv;
    }
    int32_t *row = pat + i * w;
    for (int p = 0; p < cnt; ++p) row[p] = bj[p];
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
    unsigned grid = (unsigned)((nr + KR - 1) / KR);
    if (w <= 32) knn_kernel<31><<<grid, KR, 0, s>>>(Xr, nr, d, w, pat);
    else if (w <= 64) knn_kernel<63><<<grid, KR, 0, s>>>(Xr, nr, d, w, pat);
    else if (w <= 128) knn_kernel<127><<<grid, KR, 0, s>>>(Xr, nr, d, w, pat);
    else knn_kernel<255><<<grid, KR, 0, s>>>(Xr, nr, d, w, pat);
    AFN_CUDA(cudaGetLastError());
    return AFN_OK;
}

}  // namespace afn
