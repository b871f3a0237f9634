// solve.cu -- preconditioned conjugate gradient (Alg. 5, PCG with the AFN
// apply of Alg. 3), one independent CG per right-hand-side column.
//
//  * FP64 handles: textbook PCG in FP64, x0 = 0, stop on the recursive
//    relative residual ||r|| <= tol ||b||, then the true residual is
//    recomputed and a column that is above tol restarts from its x (at most
//    3 restarts, iterations counted across restarts).
//  * Mixed handles: one FP32 PCG sequence with reliable updates (see
//    mixed_reliable): FP32 matvec / apply / vectors, FP64 scalars, x in FP64,
//    and the residual replaced by the FP64 residual b - (K + mu I) x whenever
//    the recursive one has dropped by inner_tol.  afn_options.krylov selects
//    the variants: FP64 Krylov vectors with only the matvec and the apply in
//    FP32 (AFN_KRYLOV_FP64), the same with the FP64-accurate matvec as well
//    (AFN_KRYLOV_FP64_OPERATOR), or the restarted refinement (AFN_KRYLOV_RESTART:
//    FP32 inner PCG to inner_tol, then x += d and a new FP64 residual).
//
// Scalars (rho, alpha, beta, norms) live on the device in FP64 per column.
// Each dot product is a two-level reduction whose last block sums the
// per-block partials in a fixed order and applies the scalar recurrence, so
// results are deterministic and no host round trip is needed per iteration.
// A converged column is frozen (alpha = beta = 0, no updates); the host polls
// the number of active columns every `check_every` iterations.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "afn_device.cuh"
#include "afn_internal.cuh"

namespace afn {

static constexpr int DB = 256;        // threads per dot block
static constexpr int DMAXB = 512;     // max blocks per column

enum DotMode { M_STORE = 0, M_ALPHA, M_RR, M_BETA, M_RHO0, M_NORM, M_RRU, M_SIGMA, M_BETA_PR };

struct Cols {                 // device arrays, one entry per column
    double *rho, *alpha, *beta, *val, *bnorm, *tolabs, *part;
    double *rmax2;            // largest ||r||^2 since the last residual replacement
    double *sigma;            // flexible PCG: r_{k+1}^T z_k
    int *active, *iters, *conv, *base;   // base: iters at the start of this inner solve
    int *flag;                // residual replacement requested
    unsigned int *cnt;
    int *nactive, *nflag;
};

// AFN_LOG=1 in the environment prints the refinement history to stderr
static bool log_on()
{
    static int v = -1;
    if (v < 0) {
        const char *e = getenv("AFN_LOG");
        v = (e && e[0] == '1') ? 1 : 0;
    }
    return v == 1;
}

static int dot_blocks(int64_t n)
{
    int64_t b = (n + DB * 8 - 1) / (DB * 8);
    return (int)std::max<int64_t>(1, std::min<int64_t>(b, DMAXB));
}

// out = sum_i a_i b_i per column (FP64 accumulate), then the scalar step of `mode`.
// OP 1 additionally performs x += alpha p, r -= alpha q before the r.r dot
// (a = r, b = r); for OP 1 the pointers are x, p, r, q.
template <class T, int OP>
__global__ void __launch_bounds__(DB) dot_kernel(T *a, const T *b, T *x, const T *p, int64_t n,
                                                 int64_t ld, int mode, Cols cs, int maxit)
{
    __shared__ double red[DB / 32];
    __shared__ bool last;
    const int c = blockIdx.y;
    const int nb = gridDim.x;
    const int64_t off = (int64_t)c * ld;
    double acc = 0.0;
    const bool act = cs.active[c] != 0;
    if (OP == 1) {
        if (act) {
            const double al = cs.alpha[c];
            for (int64_t i = (int64_t)blockIdx.x * DB + threadIdx.x; i < n; i += (int64_t)nb * DB) {
                T xv = x[off + i] + (T)al * p[off + i];
                T rv = a[off + i] - (T)al * b[off + i];
                x[off + i] = xv;
                a[off + i] = rv;
                acc += (double)rv * (double)rv;
            }
        } else {
            for (int64_t i = (int64_t)blockIdx.x * DB + threadIdx.x; i < n; i += (int64_t)nb * DB) {
                double rv = (double)a[off + i];
                acc += rv * rv;
            }
        }
    } else {
        for (int64_t i = (int64_t)blockIdx.x * DB + threadIdx.x; i < n; i += (int64_t)nb * DB)
            acc += (double)a[off + i] * (double)b[off + i];
    }
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < DB / 32; ++w) s += red[w];
        cs.part[(int64_t)c * DMAXB + blockIdx.x] = s;
        __threadfence();
        unsigned int prev = atomicAdd(cs.cnt + c, 1u);
        last = (prev == (unsigned)nb - 1);
    }
    __syncthreads();
    if (!last || threadIdx.x != 0) return;
    __threadfence();
    double v = 0.0;
    for (int q = 0; q < nb; ++q) v += __ldcg(cs.part + (int64_t)c * DMAXB + q);
    cs.cnt[c] = 0;
    cs.val[c] = v;
    switch (mode) {
    case M_ALPHA:
        if (act) {
            cs.alpha[c] = cs.rho[c] / v;
            cs.iters[c] += 1;
        } else {
            cs.alpha[c] = 0.0;
        }
        break;
    case M_RR:
        if (act && (sqrt(v) <= cs.tolabs[c] || cs.iters[c] - cs.base[c] >= maxit)) {
            cs.active[c] = 0;
            cs.conv[c] = sqrt(v) <= cs.tolabs[c] ? 1 : 0;
        }
        break;
    case M_BETA:
        if (act) {
            cs.beta[c] = v / cs.rho[c];
            cs.rho[c] = v;
        } else {
            cs.beta[c] = 0.0;
        }
        break;
    case M_BETA_PR:
        // flexible PCG (Polak-Ribiere form): beta = r_{k+1}^T (z_{k+1} - z_k) / rho_k
        if (act) {
            cs.beta[c] = (v - cs.sigma[c]) / cs.rho[c];
            cs.rho[c] = v;
        } else {
            cs.beta[c] = 0.0;
        }
        break;
    case M_SIGMA:
        if (act) cs.sigma[c] = v;
        break;
    case M_RHO0:
        if (act) cs.rho[c] = v;
        break;
    case M_NORM:
        cs.bnorm[c] = sqrt(v);
        break;
    case M_RRU:
        // reliable updates: ask for an FP64 residual replacement once the
        // recursive residual fell by tolabs (= delta) since the last one, or
        // when the iteration cap is reached
        if (act) {
            if (v > cs.rmax2[c]) cs.rmax2[c] = v;
            const double dl = cs.tolabs[c];
            if (v <= dl * dl * cs.rmax2[c] || cs.iters[c] - cs.base[c] >= maxit) cs.flag[c] = 1;
        }
        break;
    default:
        break;
    }
}

// p = z + beta p on active columns (beta == 0 and first == 1: p = z)
template <class T>
__global__ void pupdate_kernel(T *p, const T *z, int64_t n, int64_t ld, Cols cs, int first)
{
    const int c = blockIdx.y;
    if (!cs.active[c]) return;
    const T be = (T)cs.beta[c];
    const int64_t off = (int64_t)c * ld;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        p[off + i] = first ? z[off + i] : z[off + i] + be * p[off + i];
}

__global__ void count_active_kernel(Cols cs, int nrhs)
{
    int s = 0, f = 0;
    for (int c = 0; c < nrhs; ++c) {
        s += cs.active[c];
        f += cs.active[c] && cs.flag[c];
    }
    *cs.nactive = s;
    *cs.nflag = f;
}

// ---------------------------------------------------------- workspace --
struct Work {
    // FP64 vectors
    double *b, *x, *r, *q, *z, *p;
    // FP32 vectors (mixed)
    float *x32, *r32, *q32, *z32, *p32;
    void *tmp;          // apply temporaries
    void *mv;           // matvec scratch (FP64)
    size_t mv_bytes;
    void *mv32;
    size_t mv32_bytes;
    Cols cs, cs_out;    // inner columns / outer columns
    double *rn;         // outer residual norms
};

template <class T> static T *carve(char *&p, size_t count)
{
    T *r = reinterpret_cast<T *>(p);
    size_t bytes = (sizeof(T) * count + 255) / 256 * 256;
    p += bytes;
    return r;
}

static size_t cols_bytes(int nrhs)
{
    return (size_t)nrhs * (9 * 8 + 4 * 5 + 4) + (size_t)nrhs * DMAXB * 8 + 8 * 256 + 12288 + 256;
}

static void carve_cols(char *&p, int nrhs, Cols &cs)
{
    cs.rho = carve<double>(p, nrhs);
    cs.alpha = carve<double>(p, nrhs);
    cs.beta = carve<double>(p, nrhs);
    cs.val = carve<double>(p, nrhs);
    cs.bnorm = carve<double>(p, nrhs);
    cs.tolabs = carve<double>(p, nrhs);
    cs.part = carve<double>(p, (size_t)nrhs * DMAXB);
    cs.active = carve<int>(p, nrhs);
    cs.iters = carve<int>(p, nrhs);
    cs.conv = carve<int>(p, nrhs);
    cs.base = carve<int>(p, nrhs);
    cs.cnt = carve<unsigned int>(p, nrhs);
    cs.nactive = carve<int>(p, 1);
    cs.rmax2 = carve<double>(p, nrhs);
    cs.flag = carve<int>(p, nrhs);
    cs.nflag = carve<int>(p, 1);
    cs.sigma = carve<double>(p, nrhs);
}

static afn_status get_work(Handle *h, int nrhs, Work &wk)
{
    const int64_t n = h->n;
    const bool mixed = h->precision == AFN_PREC_MIXED;
    size_t vec64 = (size_t)n * nrhs;
    size_t need = 0;
    need += 6 * ((sizeof(double) * vec64 + 255) / 256 * 256);
    if (mixed) need += 5 * ((sizeof(float) * vec64 + 255) / 256 * 256);
    size_t tmpe = apply_tmp_elems(h, nrhs);
    need += (sizeof(double) * tmpe + 255) / 256 * 256;
    size_t mvb = matvec64_scratch(n, nrhs);
    size_t mv32b = mixed ? matvec32_scratch(n, nrhs) : 0;
    need += (mvb + 255) / 256 * 256 + (mv32b + 255) / 256 * 256;
    need += 2 * cols_bytes(nrhs) + (sizeof(double) * nrhs + 255) / 256 * 256;
    if (h->ws.bytes < need) {
        h->ws.release();
        AFN_TRY(h->ws.alloc(need));
    }
    char *p = static_cast<char *>(h->ws.p);
    wk.b = carve<double>(p, vec64);
    wk.x = carve<double>(p, vec64);
    wk.r = carve<double>(p, vec64);
    wk.q = carve<double>(p, vec64);
    wk.z = carve<double>(p, vec64);
    wk.p = carve<double>(p, vec64);
    if (mixed) {
        wk.x32 = carve<float>(p, vec64);
        wk.r32 = carve<float>(p, vec64);
        wk.q32 = carve<float>(p, vec64);
        wk.z32 = carve<float>(p, vec64);
        wk.p32 = carve<float>(p, vec64);
    } else {
        wk.x32 = wk.r32 = wk.q32 = wk.z32 = wk.p32 = nullptr;
    }
    wk.tmp = carve<double>(p, tmpe);
    wk.mv = carve<char>(p, mvb);
    wk.mv_bytes = mvb;
    wk.mv32 = mixed ? carve<char>(p, mv32b) : nullptr;
    wk.mv32_bytes = mv32b;
    char *c0 = p;
    carve_cols(p, nrhs, wk.cs);
    carve_cols(p, nrhs, wk.cs_out);
    wk.rn = carve<double>(p, nrhs);
    // the dot kernels' arrival counters (and every column field) start at
    // zero; pooled memory is reused, so clear it
    AFN_CUDA(cudaMemsetAsync(c0, 0, (size_t)(p - c0), h->stream));
    return AFN_OK;
}

// ----------------------------------------------------------- host glue --
template <class T>
static void launch_dot(int op, T *a, const T *b, T *x, const T *p, int64_t n, int nrhs, int mode,
                       const Cols &cs, int maxit, cudaStream_t s)
{
    dim3 grid(dot_blocks(n), nrhs);
    if (op == 1) dot_kernel<T, 1><<<grid, DB, 0, s>>>(a, b, x, p, n, n, mode, cs, maxit);
    else dot_kernel<T, 0><<<grid, DB, 0, s>>>(a, b, x, p, n, n, mode, cs, maxit);
}

template <class T>
static void launch_pupdate(T *p, const T *z, int64_t n, int nrhs, const Cols &cs, int first,
                           cudaStream_t s)
{
    int b = (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 1024));
    pupdate_kernel<T><<<dim3(b, nrhs), 256, 0, s>>>(p, z, n, n, cs, first);
}

static afn_status poll_active(const Cols &cs, int nrhs, cudaStream_t s, int *out)
{
    count_active_kernel<<<1, 1, 0, s>>>(cs, nrhs);
    AFN_CUDA(cudaMemcpyAsync(out, cs.nactive, sizeof(int), cudaMemcpyDeviceToHost, s));
    AFN_CUDA(cudaStreamSynchronize(s));
    return AFN_OK;
}

static afn_status apply64(Handle *h, const double *r, int nrhs, double *z, void *tmp)
{
    Scope sc(&h->prof, K_APPLY64);
    return afn_apply<double>(h, h->Linv.as<double>(), h->LinvT.as<double>(), h->Wt.as<double>(),
                             h->G.as<double>(), r, nrhs, z, static_cast<double *>(tmp), h->stream);
}

static afn_status apply32(Handle *h, const float *r, int nrhs, float *z, void *tmp)
{
    if (nrhs % 16 == 0) AFN_TRY(apply_tc_prepare(h, h->stream));
    Scope sc(&h->prof, K_APPLY32);
    return afn_apply<float>(h, h->Linv32.as<float>(), h->LinvT32.as<float>(), h->Wt32.as<float>(),
                            h->G32.as<float>(), r, nrhs, z, static_cast<float *>(tmp), h->stream);
}

// FP64-accurate q = (K + mu I) p: FP64 kernel on FP64 handles, double-float
// kernel on the FP32 pipes for mixed handles
static afn_status mv64(Handle *h, const double *p, int nrhs, double *q, const Work &wk)
{
    Scope sc(&h->prof, K_MATVEC64);
    if (h->Xdf.p)
        return matvec_df(h->Xdf.as<float2>(), h->n, stored_dim32(h->dp), h->kernel, h->mu, p, nrhs,
                         q, wk.mv, wk.mv_bytes, h->status.as<int>() + 3, h->stream);
    KParams kp{h->kernel, h->l, h->mu};
    return matvec64(h->X64.as<double>(), h->n, h->d, kp, p, nrhs, q, wk.mv, wk.mv_bytes, h->stream);
}

static afn_status mv32(Handle *h, const float *p, int nrhs, float *q, const Work &wk)
{
    Scope sc(&h->prof, K_MATVEC32);
    return matvec32(h->X32.as<float>(), h->n, h->dp, h->kernel, (float)h->mu, p, nrhs, q, wk.mv32,
                    wk.mv32_bytes, h->status.as<int>() + 3, h->stream);
}

// Generic PCG on the columns that are active in cs (x, r given; r = b - A x).
// A/M are the FP64 or FP32 operators.  Returns after every column is inactive
// or maxit iterations (per column) are reached.
template <class T>
static afn_status pcg_loop(Handle *h, const Work &wk, T *x, T *r, T *z, T *p, T *q, int nrhs,
                           int maxit)
{
    cudaStream_t s = h->stream;
    const int64_t n = h->n;
    const Cols &cs = wk.cs;
    auto A = [&](const T *pv, T *qv) -> afn_status {
        if (sizeof(T) == 8) return mv64(h, (const double *)pv, nrhs, (double *)qv, wk);
        return mv32(h, (const float *)pv, nrhs, (float *)qv, wk);
    };
    auto M = [&](const T *rv, T *zv) -> afn_status {
        if (sizeof(T) == 8) return apply64(h, (const double *)rv, nrhs, (double *)zv, wk.tmp);
        return apply32(h, (const float *)rv, nrhs, (float *)zv, wk.tmp);
    };
    AFN_TRY(M(r, z));
    {
        Scope sc(&h->prof, K_BLAS1);
        launch_dot<T>(0, r, z, nullptr, nullptr, n, nrhs, M_RHO0, cs, maxit, s);
        launch_pupdate<T>(p, z, n, nrhs, cs, 1, s);
    }
    const int every = std::max(1, h->opt.check_every);
    for (int it = 0; it < maxit; ++it) {
        AFN_TRY(A(p, q));
        {
            Scope sc(&h->prof, K_BLAS1);
            launch_dot<T>(0, p, q, nullptr, nullptr, n, nrhs, M_ALPHA, cs, maxit, s);
            launch_dot<T>(1, r, q, x, p, n, nrhs, M_RR, cs, maxit, s);
        }
        if ((it + 1) % every == 0 || it + 1 == maxit) {
            int na = 0;
            AFN_TRY(poll_active(cs, nrhs, s, &na));
            if (na == 0) break;
        }
        AFN_TRY(M(r, z));
        {
            Scope sc(&h->prof, K_BLAS1);
            launch_dot<T>(0, r, z, nullptr, nullptr, n, nrhs, M_BETA, cs, maxit, s);
            launch_pupdate<T>(p, z, n, nrhs, cs, 0, s);
        }
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "pcg launch");
    return AFN_OK;
}

// small elementwise kernels ------------------------------------------------
__global__ void residual_kernel(const double *b, const double *q, double *r, int64_t n, int nrhs)
{
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < n * nrhs) r[e] = b[e] - q[e];
}

__global__ void set_cols_kernel(Cols cs, int nrhs, double tol, const double *bn, int reset_iters)
{
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nrhs) return;
    cs.cnt[c] = 0;
    cs.tolabs[c] = tol * bn[c];
    cs.active[c] = bn[c] > 0.0 ? 1 : 0;
    cs.conv[c] = bn[c] > 0.0 ? 0 : 1;
    cs.alpha[c] = cs.beta[c] = 0.0;
    if (reset_iters) cs.iters[c] = 0;
    cs.base[c] = 0;   // FP64 PCG: max_iter caps all iterations, restarts included
}

// columns whose true relative residual is above tol become active again
__global__ void restart_cols_kernel(Cols cs, int nrhs, double tol, int maxit, const double *rn,
                                    double *relres)
{
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nrhs) return;
    double bn = cs.bnorm[c];
    double rel = bn > 0.0 ? rn[c] / bn : 0.0;
    relres[c] = rel;
    int again = (bn > 0.0) && (rel > tol) && (cs.iters[c] < maxit);
    cs.active[c] = again;
    cs.conv[c] = rel <= tol ? 1 : 0;
    cs.cnt[c] = 0;
}

__global__ void norm_from_val_kernel(const double *val, double *out, int nrhs)
{
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c < nrhs) out[c] = sqrt(val[c]);
}

// mixed: outer bookkeeping and inner set-up.  For every column with
// ||r||/||b|| > tol: r32 = r / ||r|| and inner tolerance; else inactive.
__global__ void outer_prep_kernel(Cols in, Cols out, int nrhs, double tol, double inner_tol,
                                  const double *rn, double *relres, int step, int max_outer,
                                  int maxit)
{
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nrhs) return;
    double bn = out.bnorm[c];
    double rel = bn > 0.0 ? rn[c] / bn : 0.0;
    relres[c] = rel;
    int act = (bn > 0.0) && (rel > tol) && (step < max_outer) && (in.iters[c] < maxit);
    out.active[c] = act;
    out.conv[c] = rel <= tol ? 1 : 0;
    in.active[c] = act;
    in.cnt[c] = 0;
    in.base[c] = in.iters[c];   // max_iter caps each inner solve
    in.alpha[c] = in.beta[c] = 0.0;
    // inner target: the requested inner tolerance, relaxed so that the last
    // outer step does not over-solve past what the FP64 test asks for
    double want = 0.25 * tol / (rel > 0.0 ? rel : 1.0);
    double it = inner_tol > want ? inner_tol : (want < 0.5 ? want : 0.5);
    in.tolabs[c] = it;   // ||r32|| = 1 at the start of the inner solve
}

__global__ void scale_down_kernel(const double *r, const double *rn, const int *active, float *r32,
                                  float *x32, int64_t n, int nrhs)
{
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n * nrhs) return;
    int c = (int)(e / n);
    double s = (active[c] && rn[c] > 0.0) ? 1.0 / rn[c] : 0.0;
    r32[e] = (float)(r[e] * s);
    x32[e] = 0.f;
}

__global__ void scale_up_kernel(double *x, const float *x32, const double *rn, const int *active,
                                int64_t n, int nrhs)
{
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n * nrhs) return;
    int c = (int)(e / n);
    if (active[c]) x[e] += rn[c] * (double)x32[e];
}

static unsigned g1(int64_t tot) { return (unsigned)((tot + 255) / 256); }

__global__ void init_rel_kernel(const double *bnorm, double *rel, int nrhs)
{
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c < nrhs) rel[c] = bnorm[c] > 0.0 ? 1.0 : 0.0;
}

// ----------------------------------------------- reliable-update kernels --
__global__ void ru_init_kernel(Cols cs, int nrhs, double delta)
{
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nrhs) return;
    cs.cnt[c] = 0;
    cs.tolabs[c] = delta;
    cs.flag[c] = 0;
    cs.base[c] = 0;
    cs.iters[c] = 0;
    cs.alpha[c] = cs.beta[c] = 0.0;
    cs.active[c] = cs.bnorm[c] > 0.0 ? 1 : 0;
    cs.conv[c] = cs.bnorm[c] > 0.0 ? 0 : 1;
    cs.rmax2[c] = cs.bnorm[c] * cs.bnorm[c];
}

// x64 += dx32, dx32 = 0 on active columns
__global__ void ru_accumulate_kernel(double *x, float *dx, const int *active, int64_t n, int nrhs)
{
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n * nrhs) return;
    int c = (int)(e / n);
    if (!active[c]) return;
    x[e] += (double)dx[e];
    dx[e] = 0.f;
}

__global__ void to32_kernel(const double *a, float *b, int64_t count)
{
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < count) b[e] = (float)a[e];
}

__global__ void to64_kernel(const float *a, double *b, int64_t count)
{
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < count) b[e] = (double)a[e];
}

// after a replacement: cs.val = ||b - A x||^2 (FP64); test the true residual
__global__ void ru_post_kernel(Cols cs, int nrhs, double tol, int maxit, double *relres)
{
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nrhs) return;
    double bn = cs.bnorm[c];
    double rel = bn > 0.0 ? sqrt(cs.val[c]) / bn : 0.0;
    if (!cs.active[c]) return;
    relres[c] = rel;
    cs.flag[c] = 0;
    cs.cnt[c] = 0;
    if (rel <= tol) {
        cs.active[c] = 0;
        cs.conv[c] = 1;
    } else if (cs.iters[c] >= maxit) {
        cs.active[c] = 0;
        cs.conv[c] = 0;
    } else {
        cs.rmax2[c] = cs.val[c];
    }
}

// active and flagged columns, and the status word of the staged matvec copies
static afn_status poll_both(const Cols &cs, int nrhs, const int *err, cudaStream_t s, int *na,
                            int *nf)
{
    count_active_kernel<<<1, 1, 0, s>>>(cs, nrhs);
    int h[3];
    AFN_CUDA(cudaMemcpyAsync(&h[0], cs.nactive, sizeof(int), cudaMemcpyDeviceToHost, s));
    AFN_CUDA(cudaMemcpyAsync(&h[1], cs.nflag, sizeof(int), cudaMemcpyDeviceToHost, s));
    AFN_CUDA(cudaMemcpyAsync(&h[2], err, sizeof(int), cudaMemcpyDeviceToHost, s));
    AFN_CUDA(cudaStreamSynchronize(s));
    if (h[2]) {
        set_error("FP32 matvec: a staged tile copy did not complete in time");
        return AFN_ERR_TIMEOUT;
    }
    *na = h[0];
    *nf = h[1];
    return AFN_OK;
}

// Mixed precision: one FP32 PCG sequence (FP32 matvec, apply and vectors,
// FP64 dots and scalars) whose residual is replaced by the FP64 true residual
// b - (K + mu I) x whenever the recursive residual has fallen by `delta`
// since the last replacement ("reliable updates", Sleijpen & van der Vorst
// 1996; van der Vorst & Ye 2000).  x is accumulated in FP64.  The search
// direction is kept across replacements, so the Krylov sequence is not
// restarted; convergence is declared only on the FP64 residual.
static afn_status mixed_reliable(Handle *h, Work &wk, int nrhs, double tol, int maxit,
                                 double *drel, int *steps_out)
{
    cudaStream_t s = h->stream;
    const int64_t n = h->n, tot = n * nrhs;
    const double delta = h->opt.inner_tol > 0 ? h->opt.inner_tol : 0.05;
    const bool flexible = h->opt.flexible == 1;
    const Cols &cs = wk.cs;
    ru_init_kernel<<<(nrhs + 63) / 64, 64, 0, s>>>(cs, nrhs, delta);
    AFN_CUDA(cudaMemsetAsync(wk.x, 0, sizeof(double) * tot, s));
    AFN_CUDA(cudaMemsetAsync(wk.x32, 0, sizeof(float) * tot, s));
    to32_kernel<<<g1(tot), 256, 0, s>>>(wk.b, wk.r32, tot);
    AFN_TRY(apply32(h, wk.r32, nrhs, wk.z32, wk.tmp));
    {
        Scope sc(&h->prof, K_BLAS1);
        launch_dot<float>(0, wk.r32, wk.z32, nullptr, nullptr, n, nrhs, M_RHO0, cs, maxit, s);
        launch_pupdate<float>(wk.p32, wk.z32, n, nrhs, cs, 1, s);
    }
    const int every = std::max(1, h->opt.check_every);
    int steps = 0;
    for (int it = 0; it < maxit + every; ++it) {
        AFN_TRY(mv32(h, wk.p32, nrhs, wk.q32, wk));
        {
            Scope sc(&h->prof, K_BLAS1);
            launch_dot<float>(0, wk.p32, wk.q32, nullptr, nullptr, n, nrhs, M_ALPHA, cs, maxit, s);
            launch_dot<float>(1, wk.r32, wk.q32, wk.x32, wk.p32, n, nrhs, M_RRU, cs, maxit, s);
        }
        if ((it + 1) % every == 0) {
            int na = 0, nf = 0;
            AFN_TRY(poll_both(cs, nrhs, h->status.as<int>() + 3, s, &na, &nf));
            if (na == 0) break;
            if (nf > 0) {
                // replacement for every active column: x += dx, r = b - (K + mu I) x
                ru_accumulate_kernel<<<g1(tot), 256, 0, s>>>(wk.x, wk.x32, cs.active, n, nrhs);
                AFN_TRY(mv64(h, wk.x, nrhs, wk.q, wk));
                residual_kernel<<<g1(tot), 256, 0, s>>>(wk.b, wk.q, wk.r, n, nrhs);
                launch_dot<double>(0, wk.r, wk.r, nullptr, nullptr, n, nrhs, M_STORE, cs, maxit, s);
                ru_post_kernel<<<(nrhs + 63) / 64, 64, 0, s>>>(cs, nrhs, tol, maxit, drel);
                to32_kernel<<<g1(tot), 256, 0, s>>>(wk.r, wk.r32, tot);
                ++steps;
                AFN_TRY(poll_both(cs, nrhs, h->status.as<int>() + 3, s, &na, &nf));
                if (log_on()) {
                    std::vector<double> hr(nrhs);
                    std::vector<int> hi(nrhs);
                    cudaMemcpy(hr.data(), drel, sizeof(double) * nrhs, cudaMemcpyDeviceToHost);
                    cudaMemcpy(hi.data(), cs.iters, sizeof(int) * nrhs, cudaMemcpyDeviceToHost);
                    double mx = 0;
                    int itmax = 0;
                    for (int c = 0; c < nrhs; ++c) { mx = std::max(mx, hr[c]); itmax = std::max(itmax, hi[c]); }
                    fprintf(stderr, "[afn] replacement %d: max rel. residual %.3e, iterations %d, active %d\n",
                            steps, mx, itmax, na);
                }
                if (na == 0) break;
            }
        }
        if (flexible) {
            Scope sc(&h->prof, K_BLAS1);
            launch_dot<float>(0, wk.r32, wk.z32, nullptr, nullptr, n, nrhs, M_SIGMA, cs, maxit, s);
        }
        AFN_TRY(apply32(h, wk.r32, nrhs, wk.z32, wk.tmp));
        {
            Scope sc(&h->prof, K_BLAS1);
            launch_dot<float>(0, wk.r32, wk.z32, nullptr, nullptr, n, nrhs,
                              flexible ? M_BETA_PR : M_BETA, cs, maxit, s);
            launch_pupdate<float>(wk.p32, wk.z32, n, nrhs, cs, 0, s);
        }
    }
    *steps_out = steps;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "mixed solve launch");
    return AFN_OK;
}

// The same reliable updates with the Krylov vectors in FP64: x, r, z, p, q,
// their updates and dots in FP64; only the two operators run in FP32, on
// their inputs rounded to FP32 (p for the matvec, r for the apply), their
// outputs widened back to FP64.  Rounding then enters the recurrences only
// through the operators, not through the vector updates.  exact_operator:
// the matvec too is the FP64-accurate one, so only the apply is FP32.
static afn_status mixed_reliable64(Handle *h, Work &wk, int nrhs, double tol, int maxit,
                                   double *drel, int *steps_out, bool exact_operator)
{
    cudaStream_t s = h->stream;
    const int64_t n = h->n, tot = n * nrhs;
    const double delta = h->opt.inner_tol > 0 ? h->opt.inner_tol : 0.05;
    const bool flexible = h->opt.flexible == 1;
    const Cols &cs = wk.cs;
    ru_init_kernel<<<(nrhs + 63) / 64, 64, 0, s>>>(cs, nrhs, delta);
    AFN_CUDA(cudaMemsetAsync(wk.x, 0, sizeof(double) * tot, s));
    AFN_CUDA(cudaMemcpyAsync(wk.r, wk.b, sizeof(double) * tot, cudaMemcpyDeviceToDevice, s));
    auto precondition = [&]() -> afn_status {
        to32_kernel<<<g1(tot), 256, 0, s>>>(wk.r, wk.r32, tot);
        AFN_TRY(apply32(h, wk.r32, nrhs, wk.z32, wk.tmp));
        to64_kernel<<<g1(tot), 256, 0, s>>>(wk.z32, wk.z, tot);
        return AFN_OK;
    };
    AFN_TRY(precondition());
    {
        Scope sc(&h->prof, K_BLAS1);
        launch_dot<double>(0, wk.r, wk.z, nullptr, nullptr, n, nrhs, M_RHO0, cs, maxit, s);
        launch_pupdate<double>(wk.p, wk.z, n, nrhs, cs, 1, s);
    }
    const int every = std::max(1, h->opt.check_every);
    int steps = 0;
    for (int it = 0; it < maxit + every; ++it) {
        if (exact_operator) {
            AFN_TRY(mv64(h, wk.p, nrhs, wk.q, wk));
        } else {
            to32_kernel<<<g1(tot), 256, 0, s>>>(wk.p, wk.p32, tot);
            AFN_TRY(mv32(h, wk.p32, nrhs, wk.q32, wk));
            to64_kernel<<<g1(tot), 256, 0, s>>>(wk.q32, wk.q, tot);
        }
        {
            Scope sc(&h->prof, K_BLAS1);
            launch_dot<double>(0, wk.p, wk.q, nullptr, nullptr, n, nrhs, M_ALPHA, cs, maxit, s);
            launch_dot<double>(1, wk.r, wk.q, wk.x, wk.p, n, nrhs, M_RRU, cs, maxit, s);
        }
        if ((it + 1) % every == 0) {
            int na = 0, nf = 0;
            AFN_TRY(poll_both(cs, nrhs, h->status.as<int>() + 3, s, &na, &nf));
            if (na == 0) break;
            if (nf > 0) {
                // replacement for every active column: r = b - (K + mu I) x
                AFN_TRY(mv64(h, wk.x, nrhs, wk.q, wk));
                residual_kernel<<<g1(tot), 256, 0, s>>>(wk.b, wk.q, wk.r, n, nrhs);
                launch_dot<double>(0, wk.r, wk.r, nullptr, nullptr, n, nrhs, M_STORE, cs, maxit, s);
                ru_post_kernel<<<(nrhs + 63) / 64, 64, 0, s>>>(cs, nrhs, tol, maxit, drel);
                ++steps;
                AFN_TRY(poll_both(cs, nrhs, h->status.as<int>() + 3, s, &na, &nf));
                if (na == 0) break;
            }
        }
        if (flexible) {
            Scope sc(&h->prof, K_BLAS1);
            launch_dot<double>(0, wk.r, wk.z, nullptr, nullptr, n, nrhs, M_SIGMA, cs, maxit, s);
        }
        AFN_TRY(precondition());
        {
            Scope sc(&h->prof, K_BLAS1);
            launch_dot<double>(0, wk.r, wk.z, nullptr, nullptr, n, nrhs,
                               flexible ? M_BETA_PR : M_BETA, cs, maxit, s);
            launch_pupdate<double>(wk.p, wk.z, n, nrhs, cs, 0, s);
        }
    }
    *steps_out = steps;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "mixed solve launch");
    return AFN_OK;
}

afn_status pcg_solve(Handle *h, const double *b_perm, int nrhs, double tol, double *x_perm,
                     int32_t *iters, double *relres, int *outer, int *converged)
{
    Work wk{};
    AFN_TRY(get_work(h, nrhs, wk));
    cudaStream_t s = h->stream;
    const int64_t n = h->n;
    const int64_t tot = n * nrhs;
    const int maxit = h->opt.max_iter > 0 ? h->opt.max_iter : 500;
    AFN_CUDA(cudaMemcpyAsync(wk.b, b_perm, sizeof(double) * tot, cudaMemcpyDeviceToDevice, s));
    AFN_CUDA(cudaMemsetAsync(wk.x, 0, sizeof(double) * tot, s));
    // the tensor-core kernels' timeout word starts clear for every solve
    AFN_CUDA(cudaMemsetAsync(h->status.as<int>() + 3, 0, sizeof(int), s));
    // ||b|| per column into both column sets
    launch_dot<double>(0, wk.b, wk.b, nullptr, nullptr, n, nrhs, M_NORM, wk.cs, maxit, s);
    launch_dot<double>(0, wk.b, wk.b, nullptr, nullptr, n, nrhs, M_NORM, wk.cs_out, maxit, s);
    AFN_CUDA(cudaMemsetAsync(wk.cs.iters, 0, sizeof(int) * nrhs, s));
    AFN_CUDA(cudaMemsetAsync(wk.cs_out.iters, 0, sizeof(int) * nrhs, s));
    std::vector<double> hrel(nrhs, 0.0);
    double *drel = wk.cs_out.val;   // reuse as relres staging (nrhs doubles)
    int steps = 0;
    if (h->precision != AFN_PREC_MIXED) {
        // FP64 PCG with true-residual restarts
        set_cols_kernel<<<(nrhs + 63) / 64, 64, 0, s>>>(wk.cs, nrhs, tol, wk.cs.bnorm, 1);
        AFN_CUDA(cudaMemcpyAsync(wk.r, wk.b, sizeof(double) * tot, cudaMemcpyDeviceToDevice, s));
        for (int restart = 0; restart <= 3; ++restart) {
            ++steps;
            AFN_TRY(pcg_loop<double>(h, wk, wk.x, wk.r, wk.z, wk.p, wk.q, nrhs, maxit));
            // true residual
            AFN_TRY(mv64(h, wk.x, nrhs, wk.q, wk));
            residual_kernel<<<g1(tot), 256, 0, s>>>(wk.b, wk.q, wk.r, n, nrhs);
            launch_dot<double>(0, wk.r, wk.r, nullptr, nullptr, n, nrhs, M_STORE, wk.cs_out, maxit, s);
            norm_from_val_kernel<<<(nrhs + 63) / 64, 64, 0, s>>>(wk.cs_out.val, wk.rn, nrhs);
            restart_cols_kernel<<<(nrhs + 63) / 64, 64, 0, s>>>(wk.cs, nrhs, tol, maxit, wk.rn, drel);
            int na = 0;
            AFN_TRY(poll_active(wk.cs, nrhs, s, &na));
            if (na == 0) break;
        }
        AFN_CUDA(cudaMemcpyAsync(x_perm, wk.x, sizeof(double) * tot, cudaMemcpyDeviceToDevice, s));
        AFN_CUDA(cudaMemcpyAsync(hrel.data(), drel, sizeof(double) * nrhs, cudaMemcpyDeviceToHost, s));
        if (iters) AFN_CUDA(cudaMemcpyAsync(iters, wk.cs.iters, sizeof(int) * nrhs, cudaMemcpyDeviceToHost, s));
    } else if (h->opt.krylov != AFN_KRYLOV_RESTART) {
        init_rel_kernel<<<(nrhs + 63) / 64, 64, 0, s>>>(wk.cs.bnorm, drel, nrhs);
        if (h->opt.krylov == AFN_KRYLOV_FP64 || h->opt.krylov == AFN_KRYLOV_FP64_OPERATOR)
            AFN_TRY(mixed_reliable64(h, wk, nrhs, tol, maxit, drel, &steps,
                                     h->opt.krylov == AFN_KRYLOV_FP64_OPERATOR));
        else
            AFN_TRY(mixed_reliable(h, wk, nrhs, tol, maxit, drel, &steps));
        AFN_CUDA(cudaMemcpyAsync(x_perm, wk.x, sizeof(double) * tot, cudaMemcpyDeviceToDevice, s));
        AFN_CUDA(cudaMemcpyAsync(hrel.data(), drel, sizeof(double) * nrhs, cudaMemcpyDeviceToHost, s));
        if (iters) AFN_CUDA(cudaMemcpyAsync(iters, wk.cs.iters, sizeof(int) * nrhs, cudaMemcpyDeviceToHost, s));
    } else {
        const int max_outer = h->opt.max_outer > 0 ? h->opt.max_outer : 10;
        const double inner_tol = h->opt.inner_tol > 0 ? h->opt.inner_tol : 1e-4;
        AFN_CUDA(cudaMemcpyAsync(wk.r, wk.b, sizeof(double) * tot, cudaMemcpyDeviceToDevice, s));
        for (int step = 0;; ++step) {
            // ||r|| (FP64) and outer test
            launch_dot<double>(0, wk.r, wk.r, nullptr, nullptr, n, nrhs, M_STORE, wk.cs_out, maxit, s);
            norm_from_val_kernel<<<(nrhs + 63) / 64, 64, 0, s>>>(wk.cs_out.val, wk.rn, nrhs);
            outer_prep_kernel<<<(nrhs + 63) / 64, 64, 0, s>>>(wk.cs, wk.cs_out, nrhs, tol, inner_tol,
                                                              wk.rn, drel, step, max_outer,
                                                              maxit * max_outer);
            int na = 0;
            AFN_TRY(poll_active(wk.cs_out, nrhs, s, &na));
            if (log_on()) {
                std::vector<double> hr(nrhs);
                std::vector<int> hi(nrhs);
                cudaMemcpy(hr.data(), drel, sizeof(double) * nrhs, cudaMemcpyDeviceToHost);
                cudaMemcpy(hi.data(), wk.cs.iters, sizeof(int) * nrhs, cudaMemcpyDeviceToHost);
                double mx = 0;
                int itmax = 0;
                for (int c = 0; c < nrhs; ++c) { mx = std::max(mx, hr[c]); itmax = std::max(itmax, hi[c]); }
                fprintf(stderr, "[afn] outer step %d: max rel. residual %.3e, inner iterations so far %d, active %d\n",
                        step, mx, itmax, na);
            }
            if (na == 0) break;
            ++steps;
            scale_down_kernel<<<g1(tot), 256, 0, s>>>(wk.r, wk.rn, wk.cs_out.active, wk.r32, wk.x32,
                                                     n, nrhs);
            AFN_TRY(pcg_loop<float>(h, wk, wk.x32, wk.r32, wk.z32, wk.p32, wk.q32, nrhs, maxit));
            scale_up_kernel<<<g1(tot), 256, 0, s>>>(wk.x, wk.x32, wk.rn, wk.cs_out.active, n, nrhs);
            AFN_TRY(mv64(h, wk.x, nrhs, wk.q, wk));
            residual_kernel<<<g1(tot), 256, 0, s>>>(wk.b, wk.q, wk.r, n, nrhs);
        }
        AFN_CUDA(cudaMemcpyAsync(x_perm, wk.x, sizeof(double) * tot, cudaMemcpyDeviceToDevice, s));
        AFN_CUDA(cudaMemcpyAsync(hrel.data(), drel, sizeof(double) * nrhs, cudaMemcpyDeviceToHost, s));
        if (iters) AFN_CUDA(cudaMemcpyAsync(iters, wk.cs.iters, sizeof(int) * nrhs, cudaMemcpyDeviceToHost, s));
    }
    AFN_CUDA(cudaStreamSynchronize(s));
    {
        // a bounded wait of a tensor-core kernel that ran out invalidates the solve
        int hs = 0;
        AFN_CUDA(cudaMemcpy(&hs, h->status.as<int>() + 3, sizeof(int), cudaMemcpyDeviceToHost));
        if (hs) {
            set_error("solve: a bounded device wait of a tensor-core kernel ran out");
            return AFN_ERR_TIMEOUT;
        }
    }
    int conv = 0;
    for (int c = 0; c < nrhs; ++c) {
        if (relres) relres[c] = hrel[c];
        if (hrel[c] <= tol) ++conv;
    }
    if (outer) *outer = steps;
    if (converged) *converged = conv;
    h->prof.flush();
    return conv == nrhs ? AFN_OK : AFN_ERR_NO_CONVERGE;
}

}  // namespace afn
