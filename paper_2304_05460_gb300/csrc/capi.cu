// capi.cu -- the extern "C" entry points of libafn.so (include/afn.h):
// argument checks, host/device staging, the build orchestration of Alg. 2,
// the solve (Alg. 5 with the apply of Alg. 3) and introspection.
#include <atomic>
#include <chrono>
#include <mutex>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "afn_device.cuh"
#include "afn_internal.cuh"

namespace afn {

// ------------------------------------------------------------------ errors --
static thread_local char g_err[512] = "";

void set_error(const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

afn_status cuda_fail(cudaError_t e, const char *what)
{
    set_error("CUDA error in %s: %s", what, cudaGetErrorString(e));
    if (e == cudaErrorMemoryAllocation) return AFN_ERR_OOM;
    return AFN_ERR_CUDA;
}

static thread_local cudaStream_t tl_stream = nullptr;

// limit of the bounded waits of the tcgen05 kernels (afn_set_wait_limit_ns)
static constexpr uint64_t WAIT_LIMIT_DEFAULT_NS = 2000000000ull;
static std::atomic<uint64_t> g_wait_limit_ns{WAIT_LIMIT_DEFAULT_NS};
uint64_t wait_limit_ns() { return g_wait_limit_ns.load(std::memory_order_relaxed); }

cudaStream_t current_stream() { return tl_stream; }
StreamGuard::StreamGuard(cudaStream_t s) : prev(tl_stream) { tl_stream = s; }
StreamGuard::~StreamGuard() { tl_stream = prev; }

// one pool per device; released memory stays cached in it (no automatic
// trimming: trimming happens at every synchronisation point of every thread
// once the threshold is exceeded, and stalls all concurrent streams); the
// caller returns it with afn_release_cached_memory()
static constexpr int MAX_DEV = 64;
static cudaMemPool_t g_pool[MAX_DEV];
static std::once_flag g_pool_once[MAX_DEV];

static cudaMemPool_t pool_for(int dev)
{
    if (dev < 0 || dev >= MAX_DEV) return nullptr;
    std::call_once(g_pool_once[dev], [dev]() {
        cudaMemPoolProps pr;
        memset(&pr, 0, sizeof(pr));
        pr.allocType = cudaMemAllocationTypePinned;
        pr.location.type = cudaMemLocationTypeDevice;
        pr.location.id = dev;
        cudaMemPool_t mp = nullptr;
        if (cudaMemPoolCreate(&mp, &pr) != cudaSuccess) {
            cudaGetLastError();
            mp = nullptr;
        } else {
            uint64_t keep = ~0ull;
            cudaMemPoolSetAttribute(mp, cudaMemPoolAttrReleaseThreshold, &keep);
        }
        g_pool[dev] = mp;
    });
    return g_pool[dev];
}

void trim_pool()
{
    int dev = 0;
    cudaGetDevice(&dev);
    cudaMemPool_t mp = pool_for(dev);
    if (mp) cudaMemPoolTrimTo(mp, 0);
}

afn_status DevBuf::alloc(size_t b)
{
    release();
    if (b == 0) return AFN_OK;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaMemPool_t mp = pool_for(dev);
    s = tl_stream;
    cudaError_t e = mp ? cudaMallocFromPoolAsync(&p, b, mp, s) : cudaMallocAsync(&p, b, s);
    if (e != cudaSuccess) {
        p = nullptr;
        cudaGetLastError();
        set_error("device allocation of %zu bytes failed: %s", b, cudaGetErrorString(e));
        return AFN_ERR_OOM;
    }
    bytes = b;
    return AFN_OK;
}

void DevBuf::release()
{
    if (p) cudaFreeAsync(p, s);
    p = nullptr;
    bytes = 0;
}

// --------------------------------------------------------------- profiling --
static const char *KNAMES[K_COUNT] = {"matvec32", "matvec64", "apply32", "apply64", "fps",
                                      "knn", "chol", "trsm", "fsai", "blas1", "rank"};
const char *kid_name(int k) { return (k >= 0 && k < K_COUNT) ? KNAMES[k] : "?"; }

void Profiler::begin(int, cudaEvent_t *a)
{
    if (pool.empty()) {
        cudaEvent_t e;
        cudaEventCreate(&e);
        pool.push_back(e);
    }
    *a = pool.back();
    pool.pop_back();
    cudaEventRecord(*a, s);
}

void Profiler::end(int kid, cudaEvent_t a)
{
    cudaEvent_t b;
    if (pool.empty()) cudaEventCreate(&b);
    else { b = pool.back(); pool.pop_back(); }
    cudaEventRecord(b, s);
    pending.push_back({kid, a, b});
    if (pending.size() > 4096) flush();
}

void Profiler::flush()
{
    for (auto &r : pending) {
        float ms_ = 0.f;
        cudaEventSynchronize(r.b);
        cudaEventElapsedTime(&ms_, r.a, r.b);
        count[r.kid] += 1;
        ms[r.kid] += ms_;
        pool.push_back(r.a);
        pool.push_back(r.b);
    }
    pending.clear();
}

void Profiler::reset()
{
    flush();
    for (int i = 0; i < K_COUNT; ++i) { count[i] = 0; ms[i] = 0; }
}

Profiler::~Profiler()
{
    for (auto &r : pending) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
    for (auto e : pool) cudaEventDestroy(e);
}

int64_t Handle::device_bytes() const
{
    const DevBuf *b[] = {&perm, &X64, &X32, &Xdf, &L, &Linv, &LinvT, &Linv32, &LinvT32, &Wt, &Wt32, &Wu1, &Wu2, &Wb1, &Wb2,
                         &Bn, &Bn32, &LcInv, &LcInvT, &LcInv32, &LcInvT32,
                         &pat, &G, &G32, &gt_ptr, &gt_row, &gt_slot, &gtv, &gtv32, &status, &ws};
    int64_t s = 0;
    for (auto x : b) s += (int64_t)x->bytes;
    return s;
}

double auto_rho_limit(const afn_options &o) { return o.auto_rho > 0.0 ? o.auto_rho : 0.3; }

bool is_device_ptr(const void *p)
{
    if (!p) return false;
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

afn_status sync_status(Handle *h, const char *what)
{
    AFN_CUDA(cudaStreamSynchronize(h->stream));
    int st = 0;
    AFN_CUDA(cudaMemcpyAsync(&st, h->status.p, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    AFN_CUDA(cudaStreamSynchronize(h->stream));
    if (st == DEV_NOT_SPD) {
        set_error("%s: matrix not numerically SPD", what);
        return AFN_ERR_NOT_SPD;
    }
    if (st == DEV_TIMEOUT) {
        set_error("%s: device wait exceeded its limit", what);
        return AFN_ERR_TIMEOUT;
    }
    return AFN_OK;
}

void uniform_sample_host(int64_t n, int64_t k, uint64_t seed, std::vector<int64_t> &out)
{
    // partial Fisher-Yates driven by SplitMix64 (Steele, Lea, Flood 2014)
    std::vector<int64_t> a((size_t)n);
    for (int64_t j = 0; j < n; ++j) a[(size_t)j] = j;
    uint64_t st = seed;
    out.resize((size_t)k);
    for (int64_t i = 0; i < k; ++i) {
        st += 0x9E3779B97F4A7C15ULL;
        uint64_t z = st;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
        z = z ^ (z >> 31);
        int64_t j = i + (int64_t)(z % (uint64_t)(n - i));
        std::swap(a[(size_t)i], a[(size_t)j]);
        out[(size_t)i] = a[(size_t)i];
    }
}

// finite check of a device array: any NaN/Inf sets *flag
__global__ void finite_kernel(const double *a, int64_t n, int *flag)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && !isfinite(a[i])) atomicExch(flag, 1);
}

afn_status check_finite(const double *a, int64_t count, int *dflag, cudaStream_t s,
                               const char *what)
{
    if (count <= 0) return AFN_OK;
    AFN_CUDA(cudaMemsetAsync(dflag, 0, sizeof(int), s));
    finite_kernel<<<(unsigned)((count + 255) / 256), 256, 0, s>>>(a, count, dflag);
    int hf = 0;
    AFN_CUDA(cudaMemcpyAsync(&hf, dflag, sizeof(int), cudaMemcpyDeviceToHost, s));
    AFN_CUDA(cudaStreamSynchronize(s));
    if (hf) {
        set_error("%s contains NaN or Inf", what);
        return AFN_ERR_ARG;
    }
    return AFN_OK;
}

// stage a caller buffer (host or device) as a device buffer
afn_status to_device(const double *src, int64_t count, DevBuf &tmp, const double **out,
                            cudaStream_t s)
{
    if (is_device_ptr(src)) {
        *out = src;
        return AFN_OK;
    }
    AFN_TRY(tmp.alloc(sizeof(double) * (size_t)count));
    AFN_CUDA(cudaMemcpyAsync(tmp.p, src, sizeof(double) * count, cudaMemcpyHostToDevice, s));
    *out = tmp.as<double>();
    return AFN_OK;
}

// x[:, c] gathered / scattered through perm (n x nrhs column-major)
__global__ void gather_cols_kernel(const double *__restrict__ src, const int64_t *__restrict__ perm,
                                   int64_t n, int nrhs, double *__restrict__ dst)
{
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n * nrhs) return;
    int64_t c = e / n, p = e % n;
    dst[e] = src[c * n + perm[p]];
}

__global__ void scatter_cols_kernel(const double *__restrict__ src, const int64_t *__restrict__ perm,
                                    int64_t n, int nrhs, double *__restrict__ dst)
{
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n * nrhs) return;
    int64_t c = e / n, p = e % n;
    dst[c * n + perm[p]] = src[e];
}

void gather_cols(const double *src, const int64_t *perm, int64_t n, int nrhs, double *dst,
                 cudaStream_t s)
{
    int64_t tot = n * nrhs;
    if (tot > 0)
        gather_cols_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(src, perm, n, nrhs, dst);
}

void scatter_cols(const double *src, const int64_t *perm, int64_t n, int nrhs, double *dst,
                  cudaStream_t s)
{
    int64_t tot = n * nrhs;
    if (tot > 0)
        scatter_cols_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(src, perm, n, nrhs, dst);
}

// ------------------------------------------------------------------- build --
// AFN_LOG_BUILD=1 in the environment: host wall time of each build step on
// stderr (the stream is synchronised at every mark; diagnostics only)
struct StepLog {
    bool on = false;
    const Handle *h;
    std::chrono::steady_clock::time_point t;
    explicit StepLog(const Handle *hh) : h(hh)
    {
        const char *e = getenv("AFN_LOG_BUILD");
        on = e && e[0] == '1';
        t = std::chrono::steady_clock::now();
    }
    void mark(const char *what)
    {
        if (!on) return;
        cudaStreamSynchronize(h->stream);
        const auto now = std::chrono::steady_clock::now();
        fprintf(stderr, "[afn build n=%lld d=%d] %-10s %9.1f ms\n", (long long)h->n, h->d, what,
                std::chrono::duration<double, std::milli>(now - t).count());
        t = now;
    }
};

static afn_status build_impl(Handle *h, const double *points)
{
    StepLog log(h);
    cudaStream_t s = h->stream;
    const int64_t n = h->n;
    const int d = h->d;
    KParams kp{h->kernel, h->l, h->mu};
    AFN_TRY(h->status.alloc(sizeof(int) * 4));
    AFN_CUDA(cudaMemsetAsync(h->status.p, 0, sizeof(int) * 4, s));
    int *st = h->status.as<int>();

    DevBuf pin;
    const double *X0 = nullptr;
    AFN_TRY(to_device(points, n * d, pin, &X0, s));
    AFN_TRY(check_finite(X0, n * d, st, s, "points"));
    log.mark("input");

    // k (Alg. 4 or fixed)
    int64_t k = std::min<int64_t>(h->k, n);
    if (h->opt.rank_mode == AFN_RANK_ESTIMATE || h->opt.precond == AFN_PRECOND_AUTO) {
        Scope sc(&h->prof, K_RANK);
        int64_t r = 0;
        int br = 0;
        int m = h->opt.rank_subsample > 0 ? h->opt.rank_subsample : (int)std::min<int64_t>(n, 1000);
        AFN_TRY(rank_estimate(X0, n, d, kp, m, h->opt.seed, h->k, &k, &r, &br, st, s));
        h->rank_r = r;
        h->rank_branch = br;
    }
    h->k = k;
    h->nr = n - k;
    const int64_t nr = h->nr;
    // Alg. 5: the Nystrom preconditioner when the estimated rank is below the threshold
    h->precond = h->opt.precond;
    if (h->precond == AFN_PRECOND_AUTO) {
        const int thr = h->opt.precond_threshold > 0 ? h->opt.precond_threshold : 2000;
        h->precond = k < thr ? AFN_PRECOND_NYSTROM : AFN_PRECOND_AFN;
    }
    h->w = (int)std::max<int64_t>(1, std::min<int64_t>(h->w_req, std::max<int64_t>(nr, 1)));

    // landmarks (Alg. 2: FPS when d <= 10, uniform otherwise, or forced); with the
    // maximin Schur order FPS continues over all n points and its order is the permutation
    int pol = h->opt.landmarks;
    if (pol == AFN_LM_AUTO) pol = (d <= 10) ? AFN_LM_FPS : AFN_LM_UNIFORM;
    const bool maximin = h->opt.schur_order == 1 && h->precond == AFN_PRECOND_AFN && k > 0;
    if (maximin && pol != AFN_LM_FPS) {
        set_error("schur_order = 1 (maximin) needs FPS landmarks");
        return AFN_ERR_ARG;
    }
    const int64_t kf = maximin ? n : k;     // FPS steps
    DevBuf lm;
    AFN_TRY(lm.alloc(sizeof(int64_t) * (size_t)std::max<int64_t>(kf, 1)));
    if (k > 0) {
        if (pol == AFN_LM_FPS) {
            Scope sc(&h->prof, K_FPS);
            int64_t start = h->opt.fps_start;
            if (start < 0) {
                DevBuf ds;
                AFN_TRY(ds.alloc(sizeof(int64_t)));
                AFN_TRY(centroid_start(X0, n, d, ds.as<int64_t>(), s));
                AFN_CUDA(cudaMemcpyAsync(&start, ds.p, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
                AFN_CUDA(cudaStreamSynchronize(s));
            }
            if (start >= n) {
                set_error("fps_start %lld out of range", (long long)start);
                return AFN_ERR_ARG;
            }
            AFN_TRY(fps_run(X0, n, d, kf, start, lm.as<int64_t>(), st + 1, s));
        } else {
            std::vector<int64_t> hl;
            uniform_sample_host(n, k, h->opt.seed, hl);
            AFN_CUDA(cudaMemcpyAsync(lm.p, hl.data(), sizeof(int64_t) * k, cudaMemcpyHostToDevice, s));
            AFN_CUDA(cudaStreamSynchronize(s));
        }
    }
    AFN_TRY(h->perm.alloc(sizeof(int64_t) * (size_t)n));
    log.mark("landmarks");
    AFN_TRY(build_perm(lm.as<int64_t>(), kf, n, h->perm.as<int64_t>(), s));
    AFN_TRY(h->X64.alloc(sizeof(double) * (size_t)(n * d)));
    AFN_TRY(gather_points(X0, h->perm.as<int64_t>(), n, d, h->X64.as<double>(), s));
    const double *Xk = h->X64.as<double>();
    const double *Xr = Xk + k * d;
    h->dp = pad_dim(d);
    const int ds = stored_dim32(h->dp);
    if (h->precision == AFN_PREC_MIXED || h->precision == AFN_PREC_AUTO) {
        AFN_TRY(h->X32.alloc(sizeof(float) * (size_t)(n * ds)));
        AFN_TRY(make_points32(h->X64.as<double>(), n, d, h->dp, h->kernel, h->l, h->X32.as<float>(), s));
    }
    if (h->precision == AFN_PREC_AUTO) {
        // the FP32 matvec errs by about 2^-24 sum_j K_ij |p_j|; next to mu |p_i|
        // that is at most rho = 2^-24 max_i sum_j K_ij / mu (Gershgorin bound
        // of ||K||_2 for a non-negative K)
        double rmax = 0.0;
        AFN_TRY(kernel_row_sum_max(h->X32.as<float>(), n, h->dp, h->kernel, &rmax, s));
        h->rho32 = rmax * 0x1p-24 / h->mu;
        h->precision = h->rho32 <= auto_rho_limit(h->opt) ? AFN_PREC_MIXED : AFN_PREC_DF;
        if (h->precision != AFN_PREC_MIXED) h->X32.release();
    }
    log.mark("points");
    const bool mixed = h->precision == AFN_PREC_MIXED;
    // mixed handles with FP64 factors: W and G as for an FP64 handle
    const bool f64fac = mixed && h->opt.factors == AFN_FACTORS_FP64;
    if (mixed || h->precision == AFN_PREC_DF) {
        AFN_TRY(h->Xdf.alloc(sizeof(float2) * (size_t)(n * ds)));
        AFN_TRY(make_points_df(h->X64.as<double>(), n, d, ds, h->kernel, h->l, h->Xdf.as<float2>(), s));
    }

    if (h->precond == AFN_PRECOND_NYSTROM) {
        // column-sampling Nystrom (Sec. 2): L = chol(K_SS + nu I), nu = n 2^-52, B = K(X, X_S)
        // L^{-T} for all n points, then Lc = chol(mu I + B^T B); the apply is eq.
        // (nystrom1-smw) through the SMW identity (K_nys + mu I)^{-1} = (I - B (mu I +
        // B^T B)^{-1} B^T) / mu, the same operator without an eigendecomposition
        if (k > 0) {
            {
                Scope sc(&h->prof, K_CHOL);
                AFN_TRY(h->L.alloc(sizeof(double) * (size_t)(k * k)));
                AFN_TRY(kernel_block(Xk, k, Xk, k, d, kp, (double)n * 0x1p-52, h->L.as<double>(), k, s));
                AFN_TRY(cholesky64(h->L.as<double>(), k, st, s, -1.0));
            }
            AFN_TRY(sync_status(h, "Cholesky of K_SS + nu I"));
            {
                Scope sc(&h->prof, K_TRSM);
                AFN_TRY(h->Bn.alloc(sizeof(double) * (size_t)(n * k)));
                AFN_TRY(kernel_block(Xk, n, Xk, k, d, kp, 0.0, h->Bn.as<double>(), k, s));
                AFN_TRY(trsm_right_lt64(h->L.as<double>(), k, h->Bn.as<double>(), n, s));
            }
            {
                Scope sc(&h->prof, K_CHOL);
                AFN_TRY(nystrom_factor(h, s));
            }
        }
        AFN_CUDA(cudaStreamSynchronize(s));
        log.mark("nystrom");
        return AFN_OK;
    }
    if (k > 0) {
        {
            Scope sc(&h->prof, K_CHOL);
            AFN_TRY(h->L.alloc(sizeof(double) * (size_t)(k * k)));
            AFN_TRY(kernel_block(Xk, k, Xk, k, d, kp, h->mu, h->L.as<double>(), k, s));
            AFN_TRY(cholesky64(h->L.as<double>(), k, st, s, -1.0));
        }
        AFN_TRY(sync_status(h, "Cholesky of K11 + mu I"));
        log.mark("cholesky");
        Scope sc(&h->prof, K_TRSM);
        if (!mixed || f64fac) {
            AFN_TRY(h->Linv.alloc(sizeof(double) * (size_t)(k * k)));
            AFN_TRY(h->LinvT.alloc(sizeof(double) * (size_t)(k * k)));
            AFN_TRY(tri_inverse64(h->L.as<double>(), k, h->Linv.as<double>(), h->LinvT.as<double>(), s));
            if (nr > 0) {
                // W^T = K21 L^{-T}: the kernel block, then one tiled product with the
                // triangular inverse (the same operator as the triangular solve)
                AFN_TRY(h->Wt.alloc(sizeof(double) * (size_t)(nr * k)));
                DevBuf K21;
                AFN_TRY(K21.alloc(sizeof(double) * (size_t)(nr * k)));
                AFN_TRY(kernel_block(Xr, nr, Xk, k, d, kp, 0.0, K21.as<double>(), k, s));
                // FP64 handles in FP64; double-float handles in double-float arithmetic on the
                // FP32 pipes (the same 48-bit accuracy their matvec has, far faster)
                if (h->precision == AFN_PREC_DF)
                    AFN_TRY(gemm_upper_df(K21.as<double>(), nr, k, h->LinvT.as<double>(), h->Wt.as<double>(), s));
                else
                    AFN_TRY(gemm_upper64(K21.as<double>(), nr, k, h->LinvT.as<double>(), h->Wt.as<double>(), s));
            }
            if (mixed) {
                // FP64 factors rounded to FP32 for the apply of the mixed solves
                AFN_TRY(h->Linv32.alloc(sizeof(float) * (size_t)(k * k)));
                AFN_TRY(h->LinvT32.alloc(sizeof(float) * (size_t)(k * k)));
                AFN_TRY(convert64to32(h->Linv.as<double>(), h->Linv32.as<float>(), k * k, s));
                AFN_TRY(convert64to32(h->LinvT.as<double>(), h->LinvT32.as<float>(), k * k, s));
                if (nr > 0) {
                    AFN_TRY(h->Wt32.alloc(sizeof(float) * (size_t)(nr * k)));
                    AFN_TRY(convert64to32(h->Wt.as<double>(), h->Wt32.as<float>(), nr * k, s));
                }
                AFN_CUDA(cudaStreamSynchronize(s));
                h->Linv.release();
                h->LinvT.release();
            }
        } else {
            // L^{-1} in FP64 from the FP64 factor (L is ill-conditioned when K11 is), rounded
            // once to FP32 for W and the apply
            {
                DevBuf Li, LiT;
                AFN_TRY(Li.alloc(sizeof(double) * (size_t)(k * k)));
                AFN_TRY(LiT.alloc(sizeof(double) * (size_t)(k * k)));
                AFN_TRY(tri_inverse64(h->L.as<double>(), k, Li.as<double>(), LiT.as<double>(), s));
                AFN_TRY(h->Linv32.alloc(sizeof(float) * (size_t)(k * k)));
                AFN_TRY(h->LinvT32.alloc(sizeof(float) * (size_t)(k * k)));
                AFN_TRY(convert64to32(Li.as<double>(), h->Linv32.as<float>(), k * k, s));
                AFN_TRY(convert64to32(LiT.as<double>(), h->LinvT32.as<float>(), k * k, s));
            }
            if (nr > 0) {
                // W^T = K21 L^{-T}: the kernel block, then one tiled product with the
                // triangular inverse (the same operator as the triangular solve)
                AFN_TRY(h->Wt32.alloc(sizeof(float) * (size_t)(nr * k)));
                DevBuf K21;
                AFN_TRY(K21.alloc(sizeof(float) * (size_t)(nr * k)));
                const float *X32 = h->X32.as<float>();
                AFN_TRY(kernel_block32(X32 + k * ds, nr, X32, k, h->dp, h->kernel, K21.as<float>(), k, s));
                AFN_TRY(gemm_upper32(K21.as<float>(), nr, k, h->LinvT32.as<float>(), h->Wt32.as<float>(), s));
            }
            AFN_CUDA(cudaStreamSynchronize(s));
        }
    }
    if (nr > 0) {
        const int w = h->w;
        AFN_TRY(h->pat.alloc(sizeof(int32_t) * (size_t)(nr * w)));
        {
            Scope sc(&h->prof, K_KNN);
            log.mark("W");
            AFN_TRY(knn_pattern(Xr, nr, d, w, h->pat.as<int32_t>(), s));
            log.mark("knn");
        }
        AFN_TRY(h->G.alloc(sizeof(double) * (size_t)(nr * w)));
        {
            Scope sc(&h->prof, K_FSAI);
            if (!mixed || f64fac)
                AFN_TRY((h->precision == AFN_PREC_DF ? fsai_build_df : fsai_build64)(
                    Xr, nr, d, kp, k > 0 ? h->Wt.as<double>() : nullptr, k,
                                     h->pat.as<int32_t>(), w, h->G.as<double>(), st, s));
            else
                AFN_TRY(fsai_build32(Xr, nr, d, kp, h->Wt32.as<float>(), k, h->pat.as<int32_t>(), w,
                                     h->G.as<double>(), st, s));
        }
        AFN_TRY(sync_status(h, "FSAI pattern block"));
        log.mark("fsai");
        if (mixed) {
            AFN_TRY(h->G32.alloc(sizeof(float) * (size_t)(nr * w)));
            AFN_TRY(convert64to32(h->G.as<double>(), h->G32.as<float>(), nr * w, s));
            if (f64fac) {
                // the FP64 W has served the FSAI build; the solves read its FP32 copy
                AFN_CUDA(cudaStreamSynchronize(s));
                h->Wt.release();
            }
        }
        AFN_TRY(h->gt_ptr.alloc(sizeof(int32_t) * (size_t)(nr + 1)));
        AFN_TRY(h->gt_row.alloc(sizeof(int32_t) * (size_t)(nr * w)));
        AFN_TRY(h->gt_slot.alloc(sizeof(int32_t) * (size_t)(nr * w)));
        AFN_TRY(transpose_pattern(h->pat.as<int32_t>(), nr, w, h->gt_ptr.as<int32_t>(),
                                  h->gt_row.as<int32_t>(), h->gt_slot.as<int32_t>(), s));
        AFN_TRY(make_gt_values(h, s));
    }
    AFN_CUDA(cudaStreamSynchronize(s));
    log.mark("Gt lists");
    return AFN_OK;
}

// Validates the arguments, builds the AFN factors on stream s and returns a
// new handle (the body of afn_build; also used by the batched build).
afn_status create_handle(const double *points, int64_t n, int d, int kernel, double l, double mu,
                         int k_max, int fsai_nnz, const afn_options &o, cudaStream_t s,
                         Handle **out)
{
    *out = nullptr;
    if (!points || n < 1 || d < 1 || d > 16 || (kernel != 0 && kernel != 1) || !(l > 0) ||
        !std::isfinite(l) || !(mu > 0) || !std::isfinite(mu) || k_max < 0 || fsai_nnz < 1 ||
        fsai_nnz > 128) {
        set_error("afn_build: invalid argument (n=%lld d=%d kernel=%d l=%g mu=%g k_max=%d w=%d)",
                  (long long)n, d, kernel, l, mu, k_max, fsai_nnz);
        return AFN_ERR_ARG;
    }
    if (o.factors != AFN_FACTORS_FP32 && o.factors != AFN_FACTORS_FP64) {
        set_error("bad factors %d", o.factors);
        return AFN_ERR_ARG;
    }
    if (o.schur_order != 0 && o.schur_order != 1) {
        set_error("bad schur_order %d", o.schur_order);
        return AFN_ERR_ARG;
    }
    if (o.flexible != 0 && o.flexible != 1) {
        set_error("bad flexible %d", o.flexible);
        return AFN_ERR_ARG;
    }
    if (o.krylov < AFN_KRYLOV_FP32 || o.krylov > AFN_KRYLOV_FP64_OPERATOR) {
        set_error("bad krylov %d", o.krylov);
        return AFN_ERR_ARG;
    }
    if (!(o.auto_rho >= 0.0)) {
        set_error("bad auto_rho %g", o.auto_rho);
        return AFN_ERR_ARG;
    }
    if (o.apply_tc < 0 || o.apply_tc > 2) {
        set_error("bad apply_tc %d", o.apply_tc);
        return AFN_ERR_ARG;
    }
    if (o.precond < AFN_PRECOND_AFN || o.precond > AFN_PRECOND_AUTO || o.precond_threshold < 0) {
        set_error("bad precond %d / precond_threshold %d", o.precond, o.precond_threshold);
        return AFN_ERR_ARG;
    }
    if (o.precision < AFN_PREC_FP64 || o.precision > AFN_PREC_AUTO) {
        set_error("bad precision %d", o.precision);
        return AFN_ERR_ARG;
    }
    Handle *h = new Handle();
    cudaGetDevice(&h->dev);
    h->opt = o;
    h->stream = s;
    h->prof.on = o.profile != 0;
    h->prof.s = h->stream;
    StreamGuard sg(h->stream);
    h->n = n;
    h->d = d;
    h->kernel = kernel;
    h->l = l;
    h->mu = mu;
    h->precision = o.precision;
    h->k = std::min<int64_t>(k_max, n);
    h->w_req = fsai_nnz;
    // host wall time: build_impl ends with a synchronisation of the stream
    // (no CUDA events here: event calls stall behind graph launches of other
    // threads, e.g. the serving loop's running group)
    const auto w0 = std::chrono::steady_clock::now();
    afn_status st = build_impl(h, points);
    if (st == AFN_OK) {
        h->build_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - w0).count();
        h->prof.flush();
    }
    if (st != AFN_OK) {
        delete h;
        return st;
    }
    *out = h;
    return AFN_OK;
}

// The body of afn_solve on device data: B0 (n x nrhs, original order) is
// permuted, solved by pcg_solve on the handle's stream and x scattered back
// into x_dev (original order).  Synchronises the handle's stream.
afn_status solve_handle(Handle *h, const double *B0, int nrhs, double tol, double *x_dev,
                        int32_t *iters, double *relres, int *outer, int *conv)
{
    cudaStream_t s = h->stream;
    StreamGuard sg(s);
    const int64_t n = h->n, tot = n * nrhs;
    DevBuf bp, xp;
    AFN_TRY(bp.alloc(sizeof(double) * tot));
    AFN_TRY(xp.alloc(sizeof(double) * tot));
    gather_cols(B0, h->perm.as<int64_t>(), n, nrhs, bp.as<double>(), s);
    afn_status st = pcg_solve(h, bp.as<double>(), nrhs, tol, xp.as<double>(), iters, relres, outer,
                              conv);
    if (st == AFN_OK || st == AFN_ERR_NO_CONVERGE) {
        scatter_cols(xp.as<double>(), h->perm.as<int64_t>(), n, nrhs, x_dev, s);
        cudaError_t e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_fail(e, "solve");
    }
    return st;
}

}  // namespace afn

using namespace afn;

// Every kernel launch of this library goes through __cudaLaunchKernel (the
// target of the compiler-generated <<<>>> stubs) or
// cudaLaunchCooperativeKernel; the link step wraps both (-Wl,--wrap) so that
// the library can report how many kernels it launched.
static std::atomic<long long> g_launches{0};

namespace afn {
void count_launches(long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
}  // namespace afn

extern "C" cudaError_t __real___cudaLaunchKernel(cudaKernel_t f, dim3 g, dim3 b, void **a,
                                                 size_t sm, cudaStream_t s);
extern "C" cudaError_t __wrap___cudaLaunchKernel(cudaKernel_t f, dim3 g, dim3 b, void **a,
                                                 size_t sm, cudaStream_t s)
{
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return __real___cudaLaunchKernel(f, g, b, a, sm, s);
}

extern "C" cudaError_t __real_cudaLaunchCooperativeKernel(const void *f, dim3 g, dim3 b, void **a,
                                                          size_t sm, cudaStream_t s);
extern "C" cudaError_t __wrap_cudaLaunchCooperativeKernel(const void *f, dim3 g, dim3 b, void **a,
                                                          size_t sm, cudaStream_t s)
{
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return __real_cudaLaunchCooperativeKernel(f, g, b, a, sm, s);
}

extern "C" {

int64_t afn_launch_count(void) { return (int64_t)g_launches.load(); }

void afn_release_cached_memory(void)
{
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceSynchronize();
    trim_pool();
}

void afn_default_options(afn_options *o)
{
    if (!o) return;
    memset(o, 0, sizeof(*o));
    o->precision = AFN_PREC_FP64;
    o->landmarks = AFN_LM_AUTO;
    o->rank_mode = AFN_RANK_FIXED;
    o->rank_subsample = 0;
    o->fps_start = 0;
    o->seed = 0;
    o->max_iter = 500;
    o->max_outer = 10;
    o->inner_tol = 0.01;
    o->check_every = 4;
    o->profile = 0;
    o->stream = nullptr;
    o->precond = AFN_PRECOND_AFN;
    o->precond_threshold = 0;
    o->factors = AFN_FACTORS_FP32;
    o->apply_tc = 2;
    o->flexible = 0;
    o->schur_order = 0;
    o->krylov = AFN_KRYLOV_FP32;
    o->pad_ = 0;
    o->auto_rho = 0.0;
}

const char *afn_last_error(void) { return g_err; }

void afn_set_wait_limit_ns(int64_t ns)
{
    g_wait_limit_ns.store(ns > 0 ? (uint64_t)ns : WAIT_LIMIT_DEFAULT_NS, std::memory_order_relaxed);
}

afn_status afn_build(const double *points, int64_t n, int32_t d, int32_t kernel, double l,
                     double mu, int32_t k_max, int32_t fsai_nnz, const afn_options *opt,
                     afn_handle **out)
{
    g_err[0] = 0;
    if (!out) { set_error("out is NULL"); return AFN_ERR_ARG; }
    *out = nullptr;
    afn_options o;
    afn_default_options(&o);
    if (opt) o = *opt;
    Handle *h = nullptr;
    afn_status st = create_handle(points, n, d, kernel, l, mu, k_max, fsai_nnz, o,
                                  static_cast<cudaStream_t>(o.stream), &h);
    if (st == AFN_OK) *out = reinterpret_cast<afn_handle *>(h);
    return st;
}

void afn_free(afn_handle *hh)
{
    if (!hh) return;
    Handle *h = reinterpret_cast<Handle *>(hh);
    if (h->stream) cudaStreamSynchronize(h->stream);
    else cudaDeviceSynchronize();
    delete h;
}

afn_status afn_solve(afn_handle *hh, const double *rhs, int32_t nrhs, double tol, double *x_out,
                     afn_solve_info *info)
{
    g_err[0] = 0;
    Handle *h = reinterpret_cast<Handle *>(hh);
    if (!h || !rhs || !x_out || nrhs < 1 || !(tol > 0) || !std::isfinite(tol)) {
        set_error("afn_solve: invalid argument");
        return AFN_ERR_ARG;
    }
    cudaStream_t s = h->stream;
    StreamGuard sg(s);
    const int64_t n = h->n, tot = n * nrhs;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, s);
    DevBuf bin, xo;
    const double *B0 = nullptr;
    afn_status st = to_device(rhs, tot, bin, &B0, s);
    if (st == AFN_OK) st = check_finite(B0, tot, h->status.as<int>() + 2, s, "rhs");
    std::vector<int32_t> its(nrhs, 0);
    std::vector<double> rel(nrhs, 0.0);
    int outer = 0, conv = 0;
    const bool dev = is_device_ptr(x_out);
    double *dst = x_out;
    if (st == AFN_OK && !dev) {
        st = xo.alloc(sizeof(double) * tot);
        dst = xo.as<double>();
    }
    if (st == AFN_OK) st = solve_handle(h, B0, nrhs, tol, dst, its.data(), rel.data(), &outer, &conv);
    if ((st == AFN_OK || st == AFN_ERR_NO_CONVERGE) && !dev) {
        cudaError_t e = cudaMemcpyAsync(x_out, dst, sizeof(double) * tot, cudaMemcpyDeviceToHost, s);
        if (e != cudaSuccess) st = cuda_fail(e, "copy x_out");
    }
    cudaEventRecord(e1, s);
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess && st == AFN_OK) st = cuda_fail(e, "afn_solve");
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (info) {
        if (info->iters) memcpy(info->iters, its.data(), sizeof(int32_t) * nrhs);
        if (info->relres) memcpy(info->relres, rel.data(), sizeof(double) * nrhs);
        info->outer_steps = outer;
        info->converged = conv;
        info->solve_ms = ms;
    }
    if (st == AFN_ERR_NO_CONVERGE)
        set_error("afn_solve: %d of %d columns reached tol", conv, nrhs);
    return st;
}

afn_status afn_get_build_info(const afn_handle *hh, afn_build_info *info)
{
    const Handle *h = reinterpret_cast<const Handle *>(hh);
    if (!h || !info) { set_error("NULL argument"); return AFN_ERR_ARG; }
    memset(info, 0, sizeof(*info));
    info->n = h->n;
    info->nr = h->nr;
    info->k = h->k;
    info->d = h->d;
    info->w = h->w;
    info->kernel = h->kernel;
    info->precision = h->precision;
    info->rank_r = h->rank_r;
    info->rank_branch = h->rank_branch;
    info->precond = h->precond;
    info->l = h->l;
    info->mu = h->mu;
    info->build_ms = h->build_ms;
    info->device_bytes = h->device_bytes();
    info->rho32 = h->rho32;
    return AFN_OK;
}

static afn_status copy_out(void *dst, const void *src, size_t bytes)
{
    if (bytes == 0) return AFN_OK;
    AFN_CUDA(cudaMemcpy(dst, src, bytes, cudaMemcpyDefault));
    return AFN_OK;
}

afn_status afn_get_perm(const afn_handle *hh, int64_t *perm)
{
    const Handle *h = reinterpret_cast<const Handle *>(hh);
    if (!h || !perm) { set_error("NULL argument"); return AFN_ERR_ARG; }
    return copy_out(perm, h->perm.p, sizeof(int64_t) * h->n);
}

afn_status afn_get_L(const afn_handle *hh, double *L)
{
    const Handle *h = reinterpret_cast<const Handle *>(hh);
    if (!h || !L) { set_error("NULL argument"); return AFN_ERR_ARG; }
    return copy_out(L, h->L.p, sizeof(double) * h->k * h->k);
}

afn_status afn_get_G(const afn_handle *hh, int32_t *pattern, double *values)
{
    const Handle *h = reinterpret_cast<const Handle *>(hh);
    if (!h) { set_error("NULL argument"); return AFN_ERR_ARG; }
    if (h->precond != AFN_PRECOND_AFN) { set_error("afn_get_G: not an AFN handle"); return AFN_ERR_ARG; }
    if (pattern) AFN_TRY(copy_out(pattern, h->pat.p, sizeof(int32_t) * h->nr * h->w));
    if (values) AFN_TRY(copy_out(values, h->G.p, sizeof(double) * h->nr * h->w));
    return AFN_OK;
}

afn_status afn_get_W(const afn_handle *hh, double *Wt)
{
    const Handle *h = reinterpret_cast<const Handle *>(hh);
    if (!h || !Wt) { set_error("NULL argument"); return AFN_ERR_ARG; }
    if (h->precond != AFN_PRECOND_AFN) { set_error("afn_get_W: not an AFN handle"); return AFN_ERR_ARG; }
    int64_t cnt = h->nr * h->k;
    if (cnt == 0) return AFN_OK;
    if (h->precision != AFN_PREC_MIXED) return copy_out(Wt, h->Wt.p, sizeof(double) * cnt);
    StreamGuard sg(h->stream);
    DevBuf tmp;
    AFN_TRY(tmp.alloc(sizeof(double) * cnt));
    AFN_TRY(convert32to64(h->Wt32.as<float>(), tmp.as<double>(), cnt, h->stream));
    AFN_CUDA(cudaStreamSynchronize(h->stream));
    return copy_out(Wt, tmp.p, sizeof(double) * cnt);
}

afn_status afn_apply_precond(afn_handle *hh, const double *r, int32_t nrhs, double *s_out)
{
    Handle *h = reinterpret_cast<Handle *>(hh);
    if (!h || !r || !s_out || nrhs < 1) { set_error("invalid argument"); return AFN_ERR_ARG; }
    cudaStream_t s = h->stream;
    StreamGuard sg(s);
    int64_t tot = h->n * nrhs;
    DevBuf rin, sd, tmp;
    const double *R = nullptr;
    AFN_TRY(to_device(r, tot, rin, &R, s));
    AFN_TRY(sd.alloc(sizeof(double) * tot));
    AFN_TRY(tmp.alloc(sizeof(double) * apply_tmp_elems(h, nrhs)));
    if (h->precision == AFN_PREC_MIXED) {
        // the FP32 apply of the mixed solve (tensor-core W products for 16k columns)
        DevBuf r32, s32;
        AFN_TRY(r32.alloc(sizeof(float) * tot));
        AFN_TRY(s32.alloc(sizeof(float) * tot));
        AFN_CUDA(cudaMemsetAsync(h->status.as<int>() + 3, 0, sizeof(int), s));
        AFN_TRY(convert64to32(R, r32.as<float>(), tot, s));
        if (nrhs % 16 == 0) AFN_TRY(apply_tc_prepare(h, s));
        AFN_TRY(afn_apply<float>(h, h->Linv32.as<float>(), h->LinvT32.as<float>(),
                                 h->Wt32.as<float>(), h->G32.as<float>(), r32.as<float>(), nrhs,
                                 s32.as<float>(), tmp.as<float>(), s));
        AFN_TRY(convert32to64(s32.as<float>(), sd.as<double>(), tot, s));
        AFN_CUDA(cudaStreamSynchronize(s));
        if (h->status.p) {
            int hs[4];
            AFN_CUDA(cudaMemcpyAsync(hs, h->status.p, sizeof(hs), cudaMemcpyDeviceToHost, s));
            AFN_CUDA(cudaStreamSynchronize(s));
            if (hs[3] != 0) {
                set_error("afn_apply_precond: a staged copy or MMA did not complete in time");
                return AFN_ERR_TIMEOUT;
            }
        }
        return copy_out(s_out, sd.p, sizeof(double) * tot);
    }
    AFN_TRY(afn_apply<double>(h, h->Linv.as<double>(), h->LinvT.as<double>(), h->Wt.as<double>(),
                              h->G.as<double>(), R, nrhs, sd.as<double>(), tmp.as<double>(), s));
    AFN_CUDA(cudaStreamSynchronize(s));
    return copy_out(s_out, sd.p, sizeof(double) * tot);
}

afn_status afn_get_kernel_stats(afn_handle *hh, const char *name, int64_t *count, double *ms)
{
    Handle *h = reinterpret_cast<Handle *>(hh);
    if (!h || !name) { set_error("NULL argument"); return AFN_ERR_ARG; }
    h->prof.flush();
    for (int i = 0; i < K_COUNT; ++i)
        if (strcmp(name, kid_name(i)) == 0) {
            if (count) *count = h->prof.count[i];
            if (ms) *ms = h->prof.ms[i];
            return AFN_OK;
        }
    set_error("unknown kernel name %s", name);
    return AFN_ERR_ARG;
}

afn_status afn_reset_kernel_stats(afn_handle *hh)
{
    Handle *h = reinterpret_cast<Handle *>(hh);
    if (!h) { set_error("NULL argument"); return AFN_ERR_ARG; }
    h->prof.reset();
    return AFN_OK;
}

// ------------------------------------------------------ op-level entries --
afn_status afn_kernel_matvec(const double *points, int64_t n, int32_t d, int32_t kernel, double l,
                             double mu, const double *p, int32_t nrhs, double *q,
                             int32_t precision, void *stream)
{
    g_err[0] = 0;
    if (!points || !p || !q || n < 1 || d < 1 || d > 16 || nrhs < 1 || !(l > 0) || !(mu >= 0) ||
        (kernel != 0 && kernel != 1)) {
        set_error("afn_kernel_matvec: invalid argument");
        return AFN_ERR_ARG;
    }
    if (precision != AFN_PREC_FP64 && precision != AFN_PREC_MIXED && precision != AFN_MATVEC_DF &&
        precision != AFN_MATVEC_DF_TC && precision != AFN_MATVEC_DF_CC) {
        set_error("afn_kernel_matvec: bad precision %d", precision);
        return AFN_ERR_ARG;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    StreamGuard sg(s);
    int64_t tot = n * nrhs;
    DevBuf xin, pin, qd, scratch;
    const double *X = nullptr, *P = nullptr;
    AFN_TRY(to_device(points, n * d, xin, &X, s));
    AFN_TRY(to_device(p, tot, pin, &P, s));
    bool qdev = is_device_ptr(q);
    double *Q = q;
    if (!qdev) {
        AFN_TRY(qd.alloc(sizeof(double) * tot));
        Q = qd.as<double>();
    }
    if (precision == AFN_PREC_FP64) {
        size_t sb = matvec64_scratch(n, nrhs);
        AFN_TRY(scratch.alloc(sb));
        KParams kp{kernel, l, mu};
        AFN_TRY(matvec64(X, n, d, kp, P, nrhs, Q, scratch.p, sb, s));
    } else if (precision == AFN_MATVEC_DF || precision == AFN_MATVEC_DF_TC ||
               precision == AFN_MATVEC_DF_CC) {
        const int sum = precision == AFN_MATVEC_DF_TC ? DF_SUM_TC
                        : precision == AFN_MATVEC_DF_CC ? DF_SUM_CC : DF_SUM_AUTO;
        const int ds = stored_dim32(pad_dim(d));
        DevBuf xd;
        AFN_TRY(xd.alloc(sizeof(float2) * n * ds));
        AFN_TRY(make_points_df(X, n, d, ds, kernel, l, xd.as<float2>(), s));
        size_t sb = matvecdf_scratch(n, nrhs, sum);
        AFN_TRY(scratch.alloc(sb));
        DevBuf flag;
        AFN_TRY(flag.alloc(sizeof(int)));
        AFN_CUDA(cudaMemsetAsync(flag.p, 0, sizeof(int), s));
        AFN_TRY(matvec_df(xd.as<float2>(), n, ds, kernel, mu, P, nrhs, Q, scratch.p, sb,
                          flag.as<int>(), s, sum));
        int hf = 0;
        AFN_CUDA(cudaMemcpyAsync(&hf, flag.p, sizeof(int), cudaMemcpyDeviceToHost, s));
        AFN_CUDA(cudaStreamSynchronize(s));
        if (hf) {
            set_error("afn_kernel_matvec: a bounded wait of the double-float matvec ran out");
            return AFN_ERR_TIMEOUT;
        }
    } else {
        int dp = pad_dim(d);
        int ds = stored_dim32(dp);
        DevBuf x32, p32, q32;
        AFN_TRY(x32.alloc(sizeof(float) * n * ds));
        AFN_TRY(p32.alloc(sizeof(float) * tot));
        AFN_TRY(q32.alloc(sizeof(float) * tot));
        AFN_TRY(make_points32(X, n, d, dp, kernel, l, x32.as<float>(), s));
        AFN_TRY(convert64to32(P, p32.as<float>(), tot, s));
        size_t sb = matvec32_scratch(n, nrhs);
        AFN_TRY(scratch.alloc(sb));
        DevBuf flag;
        AFN_TRY(flag.alloc(sizeof(int)));
        AFN_CUDA(cudaMemsetAsync(flag.p, 0, sizeof(int), s));
        AFN_TRY(matvec32(x32.as<float>(), n, dp, kernel, (float)mu, p32.as<float>(), nrhs,
                         q32.as<float>(), scratch.p, sb, flag.as<int>(), s));
        AFN_TRY(convert32to64(q32.as<float>(), Q, tot, s));
        int hf = 0;
        AFN_CUDA(cudaMemcpyAsync(&hf, flag.p, sizeof(int), cudaMemcpyDeviceToHost, s));
        AFN_CUDA(cudaStreamSynchronize(s));
        if (hf) {
            set_error("afn_kernel_matvec: a staged tile copy did not complete in time");
            return AFN_ERR_TIMEOUT;
        }
    }
    if (!qdev) AFN_CUDA(cudaMemcpyAsync(q, Q, sizeof(double) * tot, cudaMemcpyDeviceToHost, s));
    AFN_CUDA(cudaStreamSynchronize(s));
    return AFN_OK;
}

afn_status afn_fps(const double *points, int64_t n, int32_t d, int64_t k, int64_t start,
                   int64_t *idx, void *stream)
{
    g_err[0] = 0;
    if (!points || !idx || n < 1 || d < 1 || d > 16 || k < 0 || k > n || start < -1 || start >= n) {
        set_error("afn_fps: invalid argument");
        return AFN_ERR_ARG;
    }
    if (k == 0) return AFN_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    StreamGuard sg(s);
    DevBuf xin, id, stt;
    const double *X = nullptr;
    AFN_TRY(to_device(points, n * d, xin, &X, s));
    AFN_TRY(stt.alloc(sizeof(int) * 2));
    AFN_TRY(id.alloc(sizeof(int64_t) * k));
    if (start < 0) {
        DevBuf ds;
        AFN_TRY(ds.alloc(sizeof(int64_t)));
        AFN_TRY(centroid_start(X, n, d, ds.as<int64_t>(), s));
        AFN_CUDA(cudaMemcpyAsync(&start, ds.p, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        AFN_CUDA(cudaStreamSynchronize(s));
    }
    AFN_TRY(fps_run(X, n, d, k, start, id.as<int64_t>(), stt.as<int>(), s));
    return copy_out(idx, id.p, sizeof(int64_t) * k);
}

afn_status afn_knn_pattern(const double *xr, int64_t nr, int32_t d, int32_t w, int32_t *pattern,
                           void *stream)
{
    g_err[0] = 0;
    if (!xr || !pattern || nr < 1 || d < 1 || d > 16 || w < 1) {
        set_error("afn_knn_pattern: invalid argument");
        return AFN_ERR_ARG;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    StreamGuard sg(s);
    DevBuf xin, pd;
    const double *X = nullptr;
    AFN_TRY(to_device(xr, nr * d, xin, &X, s));
    AFN_TRY(pd.alloc(sizeof(int32_t) * nr * w));
    AFN_TRY(knn_pattern(X, nr, d, w, pd.as<int32_t>(), s));
    AFN_CUDA(cudaStreamSynchronize(s));
    return copy_out(pattern, pd.p, sizeof(int32_t) * nr * w);
}

afn_status afn_rank_estimate(const double *points, int64_t n, int32_t d, int32_t kernel, double l,
                             double mu, int32_t m, uint64_t seed, int32_t k_max, int64_t *k_out,
                             int64_t *r_out, int32_t *branch_out, void *stream)
{
    g_err[0] = 0;
    if (!points || !k_out || n < 1 || d < 1 || d > 16 || !(l > 0) || !(mu > 0) || k_max < 1 ||
        m < 0 || (kernel != 0 && kernel != 1)) {
        set_error("afn_rank_estimate: invalid argument");
        return AFN_ERR_ARG;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    StreamGuard sg(s);
    DevBuf xin, stt;
    const double *X = nullptr;
    AFN_TRY(to_device(points, n * d, xin, &X, s));
    AFN_TRY(stt.alloc(sizeof(int) * 2));
    AFN_CUDA(cudaMemsetAsync(stt.p, 0, sizeof(int) * 2, s));
    KParams kp{kernel, l, mu};
    int mm = m > 0 ? m : (int)std::min<int64_t>(n, 1000);
    int64_t r = 0;
    int br = 0;
    AFN_TRY(rank_estimate(X, n, d, kp, mm, seed, k_max, k_out, &r, &br, stt.as<int>(), s));
    if (r_out) *r_out = r;
    if (branch_out) *branch_out = br;
    return AFN_OK;
}

}  // extern "C"
