// afn_internal.cuh -- declarations shared by the CUDA translation units of
// libafn.so.  Device helpers, the handle layout and the launch wrappers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <functional>
#include <string>
#include <vector>

#include "../../include/afn.h"

namespace afn {

// ---------------------------------------------------------------- errors --
void set_error(const char *fmt, ...);
afn_status cuda_fail(cudaError_t e, const char *what);

#define AFN_CUDA(call)                                                  \
    do {                                                                \
        cudaError_t e_ = (call);                                        \
        if (e_ != cudaSuccess) return ::afn::cuda_fail(e_, #call);      \
    } while (0)

#define AFN_TRY(call)                                                   \
    do {                                                                \
        afn_status s_ = (call);                                         \
        if (s_ != AFN_OK) return s_;                                    \
    } while (0)

// limit of the bounded device-side waits of the tcgen05 kernels, ns
// (afn_set_wait_limit_ns; 2 s by default)
uint64_t wait_limit_ns();

// ---- tune.cu: the autotuner (launch parameters that never change a result)
// "sm<major><minor>x<SMs>" of the current device, the last field of every key
std::string tune_device_tag();
int log2_bucket(int64_t v);
bool tune_lookup(const std::string &key, int *choice);
void tune_store(const std::string &key, int choice);
// the cached choice for key, else (outside stream capture) time run(c) for c
// in [0, ncand) on stream s, record and return the fastest; fallback when
// timing is not possible
int tune_pick(const std::string &key, int ncand, const std::function<void(int)> &run,
              cudaStream_t s, int fallback);
// run the work once with the key's candidate: the recorded choice; else, outside
// a stream capture, the default on the key's first call and then each candidate
// on one call, timed, until the fastest is recorded (no work is repeated)
void tune_run(const std::string &key, int ncand, const std::function<void(int)> &run,
              cudaStream_t s, int fallback);

// device status word values (written by kernels, read by the host)
enum : int { DEV_OK = 0, DEV_NOT_SPD = 1, DEV_TIMEOUT = 2 };

// -------------------------------------------------------- device buffers --
// Device memory comes from a library-owned stream-ordered pool (one per
// device) that keeps released memory cached until afn_release_cached_memory.
// A buffer is allocated on the calling thread's current library stream
// (StreamGuard) and released on the same stream, so allocation and release
// never synchronise the device: independent handles built on separate
// streams run concurrently.  That stream must outlive the buffer.
struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
    cudaStream_t s = nullptr;
    afn_status alloc(size_t b);
    void release();
    ~DevBuf() { release(); }
    template <class T> T *as() const { return static_cast<T *>(p); }
};

cudaStream_t current_stream();          // the calling thread's library stream
struct StreamGuard {                    // sets it for the scope of an entry point
    cudaStream_t prev;
    explicit StreamGuard(cudaStream_t s);
    ~StreamGuard();
};
void trim_pool();                       // return cached pool memory to the device

// ------------------------------------------------------------- profiling --
enum Kid { K_MATVEC32 = 0, K_MATVEC64, K_APPLY32, K_APPLY64, K_FPS, K_KNN, K_CHOL, K_TRSM,
           K_FSAI, K_BLAS1, K_RANK, K_COUNT };
const char *kid_name(int k);

struct Profiler {
    bool on = false;
    cudaStream_t s = nullptr;
    struct Rec { int kid; cudaEvent_t a, b; };
    std::vector<Rec> pending;
    std::vector<cudaEvent_t> pool;
    int64_t count[K_COUNT] = {0};
    double ms[K_COUNT] = {0};
    void begin(int kid, cudaEvent_t *a);
    void end(int kid, cudaEvent_t a);
    void flush();     // resolve pending records (synchronizes the events)
    void reset();
    ~Profiler();
};

struct Scope {        // RAII launch timer
    Profiler *p; int kid; cudaEvent_t a = nullptr;
    Scope(Profiler *p_, int kid_) : p(p_), kid(kid_) { if (p && p->on) p->begin(kid, &a); }
    ~Scope() { if (p && p->on) p->end(kid, a); }
};

// ------------------------------------------------------------------ handle --
struct Handle {
    int dev = 0;
    cudaStream_t stream = nullptr;
    afn_options opt{};
    int64_t n = 0, k = 0, nr = 0;
    int d = 0, dp = 0, w = 0, w_req = 1, kernel = 0, precision = 0;
    double l = 1, mu = 1;
    int64_t rank_r = 0; int rank_branch = -1;
    double rho32 = 0;     // AFN_PREC_AUTO: 2^-24 max row sum of K / mu
    double build_ms = 0;

    // permuted points
    DevBuf perm;      // int64 [n]
    DevBuf X64;       // double [n*d] permuted, row-major
    DevBuf X32;       // float  [n*dp] permuted, pre-scaled for the FP32 kernel
    DevBuf Xdf;       // float2 [n*ds] permuted, pre-scaled double-float (mixed handles)
    // factors
    DevBuf L;         // double [k*k] row-major lower
    DevBuf Linv;      // double [k*k] row-major lower, L^{-1}
    DevBuf LinvT;     // double [k*k] row-major upper, L^{-T}
    DevBuf Linv32;    // float  [k*k]
    DevBuf LinvT32;   // float  [k*k]
    DevBuf Wt;        // double [nr*k]  (FP64 handles)
    DevBuf Wt32;      // float  [nr*k]  (mixed handles)
    DevBuf Wu1, Wu2;  // float tiled images of W^T and W for the tcgen05 apply (built on first use)
    DevBuf Wb1, Wb2;  // BF16 tiled images of W^T and W (apply_tc = 2, built on first use)
    // Nystrom preconditioner (precond == AFN_PRECOND_NYSTROM): L = chol(K11 + nu I),
    // B = K(X, X_S) L^{-T} (n x k row-major, permuted order), Lc = chol(mu I + B^T B)
    int precond = AFN_PRECOND_AFN;
    DevBuf Bn, Bn32;          // double / float [n*k]
    DevBuf LcInv, LcInvT;     // double [k*k] lower / upper
    DevBuf LcInv32, LcInvT32; // float  [k*k]
    bool wu_tried = false;
    DevBuf pat;       // int32 [nr*w]
    DevBuf G;         // double [nr*w]
    DevBuf G32;       // float  [nr*w]
    DevBuf gt_ptr;    // int32 [nr+1]  CSR of G^T (column c's entries, ascending row)
    DevBuf gt_row;    // int32 [nnz]
    DevBuf gt_slot;   // int32 [nnz]   index into the ELL arrays (row*w + p)
    DevBuf gtv, gtv32;  // double / float [nnz]  G's values in the order of the G^T lists
    DevBuf status;    // int [4] device status words

    // solve workspace (grown on demand)
    int ws_nrhs = 0;
    DevBuf ws;
    Profiler prof;

    int64_t device_bytes() const;
};

// ----------------------------------------------------------- util launches --
afn_status sync_status(Handle *h, const char *what);   // sync + read device status word

// pointer kind
bool is_device_ptr(const void *p);
// AFN_PREC_AUTO threshold on rho (afn_options.auto_rho, default 0.3)
double auto_rho_limit(const afn_options &o);

// the body of afn_build: validate, build on stream s, return a new handle
afn_status create_handle(const double *points, int64_t n, int d, int kernel, double l, double mu,
                         int k_max, int fsai_nnz, const afn_options &o, cudaStream_t s,
                         Handle **out);
// afn_solve on device data in original order (permute, PCG, scatter)
afn_status solve_handle(Handle *h, const double *B0, int nrhs, double tol, double *x_dev,
                        int32_t *iters, double *relres, int *outer, int *conv);
// host or device input -> device pointer (copied into tmp when on the host)
afn_status to_device(const double *src, int64_t count, DevBuf &tmp, const double **out,
                     cudaStream_t s);
afn_status check_finite(const double *a, int64_t count, int *dflag, cudaStream_t s,
                        const char *what);
// dst[c][i] = src[c][perm[i]] and its inverse, n x nrhs column-major
void gather_cols(const double *src, const int64_t *perm, int64_t n, int nrhs, double *dst,
                 cudaStream_t s);
void scatter_cols(const double *src, const int64_t *perm, int64_t n, int nrhs, double *dst,
                  cudaStream_t s);

// kernel function constants for FP64/FP32 evaluation
struct KParams {
    int kernel;       // 0 Gaussian, 1 Matern-3/2
    double l, mu;
};

// ---- matvec.cu
// q = (K + mu I) p on permuted points; p,q n x nrhs column-major (ld = n).
afn_status matvec64(const double *X, int64_t n, int d, KParams kp, const double *p, int nrhs,
                    double *q, void *scratch, size_t scratch_bytes, cudaStream_t s);
size_t matvec64_scratch(int64_t n, int nrhs);
afn_status matvec32(const float *Xs, int64_t n, int dp, int kernel, float mu, const float *p,
                    int nrhs, float *q, void *scratch, size_t scratch_bytes, int *err,
                    cudaStream_t s);   // err: device word set to DEV_TIMEOUT if a staged copy stalls
size_t matvec32_scratch(int64_t n, int nrhs);
int pad_dim(int d);
int stored_dim32(int dp);
// FP64-accurate q = (K + mu I) p from prescaled double-float points
// (make_points_df, n x ds): kernel values in double-float on the FP32 pipes;
// the sum over j exact on the tensor cores (BF16 digit splitting,
// matvec_dfu.cuh) for at least DFU_MIN_COLS columns and DFU_MIN_N points,
// else in double-float on the FP32 pipes (small systems keep the lighter
// kernel, which shares the SMs with concurrent solves).
// err: device word set to DEV_TIMEOUT if a bounded wait of the tensor-core
// kernel runs out
static constexpr int DFU_MIN_COLS = 8;
static constexpr int64_t DFU_MIN_N = 16384;
inline bool use_dfu(int64_t n, int nrhs) { return nrhs >= DFU_MIN_COLS && n >= DFU_MIN_N; }
// sum: DF_SUM_AUTO (the rule above), DF_SUM_TC (tensor cores), DF_SUM_CC (FP32 pipes)
enum : int { DF_SUM_AUTO = 0, DF_SUM_TC = 1, DF_SUM_CC = 2 };
afn_status matvec_df(const float2 *Xd, int64_t n, int ds, int kernel, double mu, const double *p,
                     int nrhs, double *q, void *scratch, size_t scratch_bytes, int *err,
                     cudaStream_t s, int sum = DF_SUM_AUTO);
size_t matvecdf_scratch(int64_t n, int nrhs, int sum);
size_t matvecdf_scratch(int64_t n, int nrhs);
afn_status make_points_df(const double *X, int64_t n, int d, int ds, int kernel, double l,
                          float2 *Xd, cudaStream_t s);
// max_i sum_j K(x_i, x_j) from the prescaled FP32 points (FP32 matvec of ones)
afn_status kernel_row_sum_max(const float *Xs, int64_t n, int dp, int kernel, double *out,
                              cudaStream_t s);
// prescaled FP32 copy of FP64 points (n x d -> n x dp)
afn_status make_points32(const double *X, int64_t n, int d, int dp, int kernel, double l,
                         float *Xs, cudaStream_t s);

// ---- fps.cu
afn_status fps_run(const double *X, int64_t n, int d, int64_t k, int64_t start, int64_t *idx,
                   int *status, cudaStream_t s);
afn_status centroid_start(const double *X, int64_t n, int d, int64_t *out, cudaStream_t s);
afn_status build_perm(const int64_t *landmarks, int64_t k, int64_t n, int64_t *perm,
                      cudaStream_t s);
afn_status gather_points(const double *X, const int64_t *perm, int64_t n, int d, double *Xp,
                         cudaStream_t s);

// ---- knn.cu
afn_status knn_pattern(const double *Xr, int64_t nr, int d, int w, int32_t *pat,
                       cudaStream_t s);

// ---- dense.cu
afn_status kernel_block(const double *Xa, int64_t na, const double *Xb, int64_t nb, int d,
                        KParams kp, double diag_shift, double *out, int64_t ld,
                        cudaStream_t s);   // out[i*ld+j] = K(a_i, b_j) (+shift on i==j)
// in place, lower; tiny < 0: error on a pivot <= 0; tiny >= 0: drop pivots <= tiny
afn_status cholesky64(double *A, int64_t k, int *status, cudaStream_t s, double tiny);
afn_status tri_inverse64(const double *L, int64_t k, double *Linv, double *LinvT, cudaStream_t s);
afn_status trsm_right_lt64(const double *L, int64_t k, double *B, int64_t m,
                           cudaStream_t s);   // B (m x k) <- B L^{-T}
// C (m x k) = A (m x k) U, U (k x k) upper triangular, FP32 row-major (tiled SGEMM)
afn_status gemm_upper32(const float *A, int64_t m, int64_t k, const float *U, float *C, cudaStream_t s);
afn_status gemm_upper64(const double *A, int64_t m, int64_t k, const double *U, double *C, cudaStream_t s);
// the same in double-float arithmetic on the FP32 pipes (double-float handles)
afn_status gemm_upper_df(const double *A, int64_t m, int64_t k, const double *U, double *C, cudaStream_t s);
afn_status kernel_block32(const float *Xa, int64_t na, const float *Xb, int64_t nb, int dp,
                          int kernel, float *out, int64_t ld, cudaStream_t s);
afn_status convert64to32(const double *a, float *b, int64_t count, cudaStream_t s);
afn_status convert32to64(const float *a, double *b, int64_t count, cudaStream_t s);

// ---- fsai.cu
afn_status fsai_build64(const double *Xr, int64_t nr, int d, KParams kp, const double *Wt,
                        int64_t k, const int32_t *pat, int w, double *G, int *status,
                        cudaStream_t s);
// the same with the Gram in double-float arithmetic on the FP32 pipes (double-float handles)
afn_status fsai_build_df(const double *Xr, int64_t nr, int d, KParams kp, const double *Wt,
                         int64_t k, const int32_t *pat, int w, double *G, int *status,
                         cudaStream_t s);
afn_status fsai_build32(const double *Xr, int64_t nr, int d, KParams kp, const float *Wt,
                        int64_t k, const int32_t *pat, int w, double *G, int *status,
                        cudaStream_t s);
afn_status transpose_pattern(const int32_t *pat, int64_t nr, int w, int32_t *ptr, int32_t *row,
                             int32_t *slot, cudaStream_t s);

// ---- apply.cu  (all vectors permuted, n x nrhs column-major, ld = n)
template <class T>
afn_status afn_apply(const Handle *h, const T *Linv, const T *LinvT, const T *Wt, const T *G,
                     const T *r, int nrhs, T *s, T *tmp, cudaStream_t st);
size_t apply_tmp_elems(const Handle *h, int nrhs);
// tiled images of W for the tcgen05 apply of a mixed handle (no-op when they
// exist, the handle has no W, or its option apply_tc is 0)
afn_status apply_tc_prepare(Handle *h, cudaStream_t s);
// the values of G (and of its FP32 copy) in the order of the G^T column lists
afn_status make_gt_values(Handle *h, cudaStream_t s);
// the Nystrom factors of a handle whose L (chol(K11 + nu I)) and Bn are set:
// Lc = chol(mu I + B^T B) and its triangular inverses (FP32 copies for mixed
// handles)
afn_status nystrom_factor(Handle *h, cudaStream_t s);

// ---- grouped steps (many systems per launch; group.cuh describes the group)
struct GDev;
// share: fraction of each SM's CTA slots the persistent grids take (1 = all;
// less leaves room for work on other streams, e.g. the server's builds)
// cps: persistent CTAs per SM (0 = the default; the autotuner's choice)
afn_status group_matvec32(const GDev *gd, cudaStream_t s, double share, int cps = 0);
afn_status group_matvec64(const GDev *gd, cudaStream_t s, double share);
afn_status group_apply(const GDev *gd, cudaStream_t s, double share, int cps = 0);
int persistent_grid(int ctas_per_sm, double share);   // max(1, SMs x ctas_per_sm x share)
// caps, for the calling thread's scope, the fraction of CTA slots a
// double-float matvec may take (read at every launch; 1 = no cap); used by
// one-at-a-time solves running beside a group, whose owner lowers the share
// while the group has work and raises it to 1 when it has none
struct GridShareGuard {
    const std::atomic<double> *prev;
    explicit GridShareGuard(const std::atomic<double> *share);
    ~GridShareGuard();
};
int group_mv32_rows();      // rows per tile of the grouped FP32 matvec
int group_npad(int64_t n);  // n rounded up to the staged point tile
// duplicated (x, x) FP32 pairs of the prescaled points, ds + 2 per row, npad rows
void dup_points(const float *Xs, int64_t n, int ds, int64_t npad, void *Xdup, cudaStream_t s);
int group_mv64_rows();      // rows per tile of the grouped FP64 matvec
int group_block_rows();     // rows per block of the grouped dense products
int group_sparse_rows();    // rows per block of the grouped sparse products

// ---- solve.cu (PCG vector kernels; FP64 scalars per column)
afn_status pcg_solve(Handle *h, const double *b_perm, int nrhs, double tol, double *x_perm,
                     int32_t *iters, double *relres, int *outer, int *converged);

// ---- rank.cu
afn_status rank_estimate(const double *X, int64_t n, int d, KParams kp, int m, uint64_t seed,
                         int64_t k_max, int64_t *k_out, int64_t *r_out, int *branch_out,
                         int *status, cudaStream_t s);

// host SplitMix64 partial Fisher-Yates (uniform sampling without replacement)
void uniform_sample_host(int64_t n, int64_t k, uint64_t seed, std::vector<int64_t> &out);

}  // namespace afn
