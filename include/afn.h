/*
 * afn.h -- C ABI of the GB300 (sm_103a) AFN-preconditioned CG library.
 *
 * Solves the regularized kernel system (K + mu I) a = b   (eq. (Problem),
 * Sec. 1) for the Gaussian kernel exp(-||x-y||^2 / l^2) (eq. (gaussianf)) and
 * the Matern-3/2 kernel (1 + sqrt3 r/l) exp(-sqrt3 r/l) (Sec. 5), with PCG
 * preconditioned by the Adaptive Factorized Nystrom (AFN) preconditioner:
 *   landmarks X_k by farthest point sampling (Alg. 6) or uniform sampling,
 *   L = chol(K11 + mu I), G = FSAI of the Schur complement
 *   K22 + mu I - K12^T (K11 + mu I)^{-1} K12 (Alg. 1, Alg. 2),
 *   applied as in Alg. 3; the landmark count can be estimated by Alg. 4.
 *
 * Conventions shared by every entry point
 *  - Points are n x d row-major float64.  Right-hand sides and solutions are
 *    n x nrhs column-major float64 in the caller's ORIGINAL point order
 *    (the library permutes internally: landmarks first, Sec. 2).
 *  - Any pointer may be host or device memory (CUDA unified addressing
 *    decides); device pointers must be on the current device.  Inputs are
 *    read-only and fully consumed before the call returns; outputs are
 *    caller-owned.  Host outputs are valid when the call returns; device
 *    outputs are valid once the call's stream has reached that point (every
 *    call below synchronises its stream before returning, so they are valid
 *    on return as well).
 *  - Every function returns an afn_status; nothing aborts.  The message of
 *    the last failure on the calling thread is afn_last_error().
 *  - A handle is not thread-safe; distinct handles are independent.
 *  - stream: a cudaStream_t passed as void*; NULL = the legacy default stream.
 */
#ifndef AFN_H
#define AFN_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    AFN_OK = 0,
    AFN_ERR_ARG = 1,           /* invalid argument (sizes, l<=0, mu<=0, tol<=0, NaN/Inf input) */
    AFN_ERR_OOM = 2,           /* device allocation failed / admission refused */
    AFN_ERR_NOT_SPD = 3,       /* K11 + mu I or an FSAI pattern block is not numerically SPD */
    AFN_ERR_NO_CONVERGE = 4,   /* max_iter / max_outer reached; the partial result is returned */
    AFN_ERR_TIMEOUT = 5,       /* a device-side wait ran past its limit; results invalid */
    AFN_ERR_CUDA = 6,          /* a CUDA runtime error */
    AFN_ERR_BUSY = 7           /* server queue full */
} afn_status;

typedef enum { AFN_GAUSSIAN = 0, AFN_MATERN32 = 1 } afn_kernel;

typedef enum {
    AFN_PREC_FP64 = 0,         /* everything in FP64 */
    AFN_PREC_MIXED = 1,        /* FP32 matvec / apply / FSAI build + FP64 Cholesky, dots,
                                  scalars and FP64 residual replacements (reliable updates) */
    AFN_PREC_DF = 2,           /* FP64 PCG and apply; FP64-accurate factors (Cholesky and
                                  triangular inverse in FP64, W and the FSAI Gram in
                                  double-float on the FP32 pipes); the matvec FP64-accurate
                                  in double-float (its sum over j exact on the tensor cores
                                  from 8 columns and 16384 points) */
    AFN_PREC_AUTO = 3          /* per system at build time: MIXED when
                                  rho = 2^-24 max_i sum_j K_ij / mu <= 0.3 (the FP32 matvec
                                  error stays small next to mu; the option auto_rho
                                  overrides 0.3), else DF; the handle reports
                                  the precision chosen and rho (afn_build_info) */
} afn_precision;

typedef enum {
    AFN_LM_AUTO = 0,           /* FPS when d <= 10, else uniform (Alg. 2) */
    AFN_LM_FPS = 1,            /* farthest point sampling (Alg. 6) */
    AFN_LM_UNIFORM = 2         /* uniform sampling without replacement */
} afn_landmark_policy;

typedef enum {
    AFN_RANK_FIXED = 0,        /* k = min(k_max, n) */
    AFN_RANK_ESTIMATE = 1      /* k = Alg. 4 estimate clipped to [1, min(k_max, n)] */
} afn_rank_mode;

typedef enum {
    AFN_PRECOND_AFN = 0,       /* the AFN preconditioner (Alg. 2, applied by Alg. 3) */
    AFN_PRECOND_NYSTROM = 1,   /* the column-sampling Nystrom preconditioner (Sec. 2), applied
                                  as eq. (nystrom1-smw): (K_nys + mu I)^{-1} */
    AFN_PRECOND_AUTO = 2       /* Alg. 5: estimate k by Alg. 4 (rank_mode is then taken as
                                  AFN_RANK_ESTIMATE); Nystrom with k landmarks when
                                  k < precond_threshold, else AFN */
} afn_precond;

typedef struct {
    int32_t precision;         /* afn_precision, default AFN_PREC_FP64 */
    int32_t landmarks;         /* afn_landmark_policy, default AFN_LM_AUTO */
    int32_t rank_mode;         /* afn_rank_mode, default AFN_RANK_FIXED */
    int32_t rank_subsample;    /* m of Alg. 4; 0 = min(n, 1000) */
    int64_t fps_start;         /* FPS start index; -1 = the point nearest the centroid (Alg. 6) */
    uint64_t seed;             /* SplitMix64 seed for uniform landmarks and Alg. 4's subsample */
    int32_t max_iter;          /* PCG iteration cap per column (FP64) / per inner solve; default 500 */
    int32_t max_outer;         /* mixed precision, restarted refinement only
                                  (krylov = AFN_KRYLOV_RESTART): FP64 refinement steps cap;
                                  default 10 */
    double inner_tol;          /* mixed precision: drop of the FP32 recursive residual between
                                  two FP64 residual replacements (delta); default 0.01 */
    int32_t check_every;       /* iterations between host convergence polls; default 4 */
    int32_t profile;           /* 1 = time every launch with CUDA events (afn_get_kernel_stats) */
    void *stream;              /* cudaStream_t; NULL = default stream */
    int32_t precond;           /* afn_precond, default AFN_PRECOND_AFN; the batched and
                                  served solves take AFN only */
    int32_t precond_threshold; /* Alg. 5's rank threshold; 0 = 2000 */
    int32_t factors;           /* mixed handles: arithmetic of the factor build (afn_factors),
                                  default AFN_FACTORS_FP32 */
    int32_t apply_tc;          /* mixed handles: the two W products of the apply (Alg. 3) when
                                  the column count is a multiple of 16: 0 = CUDA-core FP32
                                  tiles; 1 = tcgen05 tensor cores, three-pass tf32 on the FP32
                                  W with FP32 accumulation; 2 = tcgen05 tensor cores on a BF16
                                  copy of W (half the bytes streamed), the vectors split into
                                  three BF16 terms, FP32 accumulation; default 2 */
    int32_t flexible;          /* mixed handles: 1 = flexible PCG, beta in the Polak-Ribiere
                                  form r_{k+1}^T (z_{k+1} - z_k) / r_k^T z_k (Notay 2000), which
                                  tolerates the FP32 apply being inexact; 0 = the textbook
                                  Fletcher-Reeves beta; default 0 */
    int32_t schur_order;       /* order of the Schur rows X_r, which defines "numbered less
                                  than i" of the FSAI pattern (Sec. 3.1): 0 = ascending original
                                  index; 1 = maximin, farthest point sampling continued over
                                  all n points after the k landmarks (the screening-effect
                                  ordering, Sec. 3.1; needs FPS landmarks); default 0 */
    int32_t krylov;            /* mixed handles: the Krylov scheme around the FP32 matvec and
                                  apply (afn_krylov), default AFN_KRYLOV_FP32 */
    int32_t pad_;              /* reserved, 0 */
    double auto_rho;           /* AFN_PREC_AUTO: the largest rho32 that still takes MIXED;
                                  0 = 0.3 */
} afn_options;

typedef enum {
    AFN_KRYLOV_FP32 = 0,       /* one PCG sequence with FP32 vectors (FP64 dots and scalars) and
                                  reliable updates: the residual replaced by the FP64-accurate
                                  b - (K + mu I) x once the recursive one fell by inner_tol */
    AFN_KRYLOV_FP64 = 1,       /* the same reliable updates with FP64 vectors: x, r, z, p, q
                                  and their updates in FP64, only the matvec and the apply in
                                  FP32 (their inputs rounded to FP32, outputs widened) */
    AFN_KRYLOV_RESTART = 2,    /* restarted refinement: FP32 PCG on the scaled FP64 residual to
                                  inner_tol, x updated in FP64, at most max_outer restarts */
    AFN_KRYLOV_FP64_OPERATOR = 3  /* FP64 vectors and the FP64-accurate (double-float) matvec in
                                  every iteration, only the preconditioner apply in FP32
                                  (mixed-precision preconditioning); slower per iteration,
                                  for comparison */
} afn_krylov;

typedef enum {
    AFN_FACTORS_FP32 = 0,      /* L^{-1} formed in FP64 and rounded once to FP32; K12 from the
                                  FP32 points and W = L^{-1} K12 by an FP32 product; FSAI Schur
                                  blocks with an FP32 Gram (Alg. 1) */
    AFN_FACTORS_FP64 = 1       /* W, the triangular inverses and G built in FP64 as for an FP64
                                  handle (G within the FP64 parity bound of the oracle's), then
                                  rounded to FP32 for the apply */
} afn_factors;

typedef struct afn_handle afn_handle;   /* opaque; owns every device buffer of one system */

typedef struct {
    int64_t n, nr, k;          /* points, Schur rows n-k, landmarks */
    int32_t d, w;              /* dimension, FSAI nonzeros per row (incl. diagonal) */
    int32_t kernel, precision;
    int64_t rank_r;            /* Alg. 4: the subsample Nystrom rank r (0 if not estimated) */
    int32_t rank_branch;       /* Alg. 4: 0 = k from r n / m, 1 = eigenvalue count, -1 = fixed k */
    int32_t precond;           /* afn_precond built (AFN or NYSTROM) */
    double l, mu;
    double build_ms;           /* wall time of the build (it ends synchronised) */
    int64_t device_bytes;      /* device memory held by the handle */
    double rho32;              /* AFN_PREC_AUTO: 2^-24 max_i sum_j K_ij / mu (0 otherwise) */
} afn_build_info;

typedef struct {
    int32_t *iters;            /* [nrhs] or NULL: PCG iterations per column (mixed: inner iterations summed) */
    double *relres;            /* [nrhs] or NULL: final ||b - (K+mu I)x|| / ||b|| per column, FP64 */
    int32_t outer_steps;       /* out: FP64 residual evaluations (mixed) / PCG restarts + 1 (FP64) */
    int32_t converged;         /* out: columns whose FP64 relative residual is <= tol */
    double solve_ms;           /* out: device time of the solve */
} afn_solve_info;

/* Fill *opt with the defaults listed above. */
void afn_default_options(afn_options *opt);

/*
 * Build the AFN preconditioner for points (n x d), Alg. 2:
 *   k = min(k_max, n) or the Alg. 4 estimate; landmarks by FPS (Alg. 6) or
 *   uniform sampling; L = chol(K11 + mu I); W = L^{-1} K12; FSAI pattern of
 *   each Schur row = its fsai_nnz-1 nearest lower-numbered neighbours plus
 *   itself (Sec. 3.1); G = FSAI of the Schur complement (Alg. 1).
 * kernel: afn_kernel.  l > 0, mu > 0, k_max >= 0, 1 <= fsai_nnz <= 128
 * (clamped to n - k).  opt may be NULL (defaults).  On success *out owns all device state.
 * Errors: AFN_ERR_ARG, AFN_ERR_OOM, AFN_ERR_NOT_SPD, AFN_ERR_TIMEOUT, AFN_ERR_CUDA.
 */
afn_status afn_build(const double *points, int64_t n, int32_t d, int32_t kernel, double l,
                     double mu, int32_t k_max, int32_t fsai_nnz, const afn_options *opt,
                     afn_handle **out);

/*
 * Solve (K + mu I) x = rhs for nrhs columns with AFN-PCG (Alg. 3, Alg. 5),
 * relative residual tol on each column (||r||_2 <= tol ||b||_2).  FP64 mode:
 * textbook PCG, then the true residual is recomputed and PCG restarts from x
 * while it is above tol (at most 3 restarts).  Mixed mode: one FP32 PCG
 * sequence (FP32 matvec, apply and vectors; FP64 dots and scalars) whose
 * residual is replaced by the FP64 residual b - (K + mu I) x (x kept in FP64)
 * each time the recursive residual has dropped by inner_tol; a column stops
 * when its FP64 residual is <= tol.
 * rhs, x_out: n x nrhs column-major, original point order.  info may be NULL.
 * Errors: AFN_ERR_ARG, AFN_ERR_OOM, AFN_ERR_NO_CONVERGE (x_out holds the last
 * iterate), AFN_ERR_CUDA.
 */
afn_status afn_solve(afn_handle *h, const double *rhs, int32_t nrhs, double tol, double *x_out,
                     afn_solve_info *info);

/* Release every device buffer of h.  NULL-safe. */
void afn_free(afn_handle *h);

/* Message of the last failure on this thread ("" if none). */
const char *afn_last_error(void);

/* ---- introspection of a built handle (parity checks, tooling) ---------- */
afn_status afn_get_build_info(const afn_handle *h, afn_build_info *info);
/* perm[n]: original index of the point at permuted position p (landmarks first). */
afn_status afn_get_perm(const afn_handle *h, int64_t *perm);
/* L: k x k row-major, lower triangle (upper zero), FP64. */
afn_status afn_get_L(const afn_handle *h, double *L);
/* pattern: nr x w int32 (-1 padding; diagonal last), values: nr x w FP64 (ELL of G). */
afn_status afn_get_G(const afn_handle *h, int32_t *pattern, double *values);
/* W = L^{-1} K12 as nr x k row-major (row j = column j of W), FP64 or the
 * precision the handle keeps (FP64 handle: FP64; mixed: FP32 converted). */
afn_status afn_get_W(const afn_handle *h, double *Wt);
/* s = M^{-1} r for nrhs columns (Alg. 3), vectors in PERMUTED order, FP64 in
 * and out.  FP64 handles apply in FP64; mixed handles run the FP32 apply of
 * their solves (r rounded to FP32; with the handle's option apply_tc = 1 or
 * 2, the default, and a multiple of 16 columns the W products run on the
 * tensor cores).
 * AFN_ERR_TIMEOUT if a staged copy or MMA did not complete. */
afn_status afn_apply_precond(afn_handle *h, const double *r, int32_t nrhs, double *s);

/* per-kernel timing gathered while opt.profile was set (CUDA events on the
 * launching stream).  name: "matvec32", "matvec64", "apply32", "apply64",
 * "fps", "knn", "chol", "trsm", "fsai", "blas1", "rank".  count = launches,
 * ms = total device time.  afn_reset_kernel_stats clears the counters. */
afn_status afn_get_kernel_stats(afn_handle *h, const char *name, int64_t *count, double *ms);
afn_status afn_reset_kernel_stats(afn_handle *h);

/* Number of CUDA kernels this library has launched in this process so far
 * (all entry points, all devices).  Tooling; no paper counterpart. */
int64_t afn_launch_count(void);

/* Device memory of every handle, batch and server comes from a pool owned by
 * the library (one per device) that keeps released memory cached for reuse
 * (allocation and release then never synchronise the device).  This call
 * waits for the current device to go idle and returns the cached memory to
 * the device.  No paper counterpart. */
void afn_release_cached_memory(void);

/* Limit, in nanoseconds, of the bounded device-side waits of the tensor-core
 * (tcgen05) kernels: the FP32 kernel matvec with 16, 32 or 64 columns a
 * piece, the tensor-core sum of the double-float matvec and the tensor-core
 * W products of the FP32 apply (tf32 and BF16).  A wait that runs past
 * it (a staged copy or an MMA that has not completed) raises the kernel's
 * abort flag; the kernel then still waits, up to 2 s, for the copies and
 * MMAs it has in flight, releases its tensor memory and returns, and the
 * entry point that launched it returns AFN_ERR_TIMEOUT with its results
 * invalid.  ns <= 0 restores the default, 2 s.  Process-wide; takes effect at
 * the next launch.  For testing the failure path (a limit of a few
 * nanoseconds makes the waits run out on a healthy GPU).  No paper
 * counterpart. */
void afn_set_wait_limit_ns(int64_t ns);

/* ---- the autotuner ------------------------------------------------------
 * Launch parameters that change only how work is spread over the GPU, never
 * a result (row warps per TMEM lane quarter of the tcgen05 matvec, CTAs per
 * SM of the persistent grouped kernels, threads per CTA of the FSAI build),
 * are picked by timing: the first call with a given shape times every
 * candidate on its own operands and records the fastest under a key
 * "<kernel>/<shape fields>/sm<cc>x<SMs>"; later calls reuse it.  Every
 * candidate computes the same bits, so results never depend on the choice.
 * No timing happens while the stream is being captured (the default is used
 * and not recorded).  No paper counterpart. */
/* Persist the cache in a text file ("key choice" per line): entries already
 * in the file are loaded (and override those in memory), and the file is
 * rewritten after every new decision.  NULL or "" stops persisting.
 * Errors: AFN_ERR_ARG (unreadable or malformed file, unwritable path). */
afn_status afn_tune_set_cache(const char *path);
/* The recorded choice for key; AFN_ERR_ARG when there is none. */
afn_status afn_tune_get(const char *key, int32_t *choice);
/* Record a choice (key: printable, no spaces, at most 200 characters;
 * choice >= 0); the library uses it from then on.  A choice outside the
 * key's candidates (here or in a loaded file) is ignored: the key is tuned
 * again and the entry replaced.  Errors: AFN_ERR_ARG. */
afn_status afn_tune_put(const char *key, int32_t choice);
/* Entries in the cache; the key of entry index (sorted order) copied into
 * buf (len bytes, NUL-terminated) and its choice returned, -1 past the end. */
int32_t afn_tune_count(void);
int32_t afn_tune_key(int32_t index, char *buf, int32_t len);
/* Forget every entry (and empty the persisted file, if any). */
void afn_tune_clear(void);

/* ---- operator-level entry points (each one step of the hot path) ------- */

/*
 * q = (K + mu I) p, matrix-free (eq. (Problem); K_ij = K(x_i, x_j), Sec. 1).
 * points n x d row-major FP64; p, q n x nrhs column-major FP64.  precision:
 * AFN_PREC_FP64 computes in FP64; AFN_PREC_MIXED evaluates pairs in FP32
 * (points and p rounded to FP32, FP32 accumulation) and returns FP64;
 * AFN_PREC_DF computes FP64-accurate values (kernel values in double-float
 * on the FP32 pipes, within 2e-14 absolute; Gaussian values above 2^-100
 * within 2e-14 relative) -- the kernel of the DF solves and of the
 * mixed solves' FP64 residual b - (K + mu I) x: with at least 8 columns and
 * 16384 points the sum over j runs exactly on the tensor cores (both
 * operands split into BF16 base-256 digits, integer products accumulated
 * exactly in FP32; Ozaki et al. 2012), otherwise in double-float on the FP32
 * pipes.  AFN_MATVEC_DF_TC takes the tensor-core sum at every size (each
 * column of p scaled by its own power of two, so columns of any magnitude);
 * AFN_MATVEC_DF_CC the double-float sum at every size.
 */
#define AFN_MATVEC_DF AFN_PREC_DF
#define AFN_MATVEC_DF_TC 4
#define AFN_MATVEC_DF_CC 5
afn_status afn_kernel_matvec(const double *points, int64_t n, int32_t d, int32_t kernel, double l,
                             double mu, const double *p, int32_t nrhs, double *q,
                             int32_t precision, void *stream);

/*
 * afn_kernel_matvec_noalloc: the FP64 q = (K + mu I) p of afn_kernel_matvec
 * for callers that cannot allocate device memory: services whose device
 * memory is planned up front and handed out by their own pool (an allocation
 * outside it breaks the plan, or fails once the pool holds the rest of the
 * device), and plug-ins that must not grow the host process's device
 * footprint.  The paper has no counterpart; this is an interface convenience.
 *  - points (n x d row-major), p and q (n x nrhs column-major) must all be
 *    device memory on the current device; nothing is staged or allocated.
 *  - The split-K partial sums live in a fixed 16 MiB __device__ array built
 *    into the library (held by every GPU that loads it until exit).  Columns
 *    are processed in groups of up to 8 that fit it; a size whose single
 *    column does not fit (n above roughly 2 million) is rejected with
 *    AFN_ERR_ARG and a message naming the bytes needed.
 *  - The first call on a device looks up the array's device address
 *    (cudaGetSymbolAddress) with that device current; make it before any
 *    stream capture.
 *  - All calls share the array: calls whose kernels overlap on the GPU (on
 *    streams with no ordering between them) race.  Calls in order on one
 *    stream are safe; nothing needs zeroing between calls.
 * Synchronises `stream` before returning.  Errors: AFN_ERR_ARG, AFN_ERR_CUDA.
 */
afn_status afn_kernel_matvec_noalloc(const double *points, int64_t n, int32_t d, int32_t kernel,
                                     double l, double mu, const double *p, int32_t nrhs,
                                     double *q, void *stream);

/*
 * Farthest point sampling, Alg. 6: idx[0] = start (or the point nearest the
 * centroid when start == -1), then k-1 times the point with the largest
 * squared distance (FP64, summed over dimensions in order, no fused
 * multiply-add) to the selected set; ties go to the lowest index; a selected
 * point is never selected again.  idx: k int64.
 */
afn_status afn_fps(const double *points, int64_t n, int32_t d, int64_t k, int64_t start,
                   int64_t *idx, void *stream);

/*
 * FSAI pattern (Sec. 3.1) of the point sequence xr (nr x d): row i lists the
 * w-1 nearest points j < i by (FP64 squared distance, j) ascending, then i
 * itself; rows with i < w-1 list all j < i.  pattern: nr x w int32, -1 padded.
 */
afn_status afn_knn_pattern(const double *xr, int64_t nr, int32_t d, int32_t w, int32_t *pattern,
                           void *stream);

/*
 * Alg. 4 rank estimate (readings: subsample = first m SplitMix64 partial
 * Fisher-Yates draws with `seed`; FPS from subsample index 0; error of rank r
 * = ||E_r||_2 / ||K_m||_2 with E_r the Schur complement after r FPS pivots;
 * r = smallest rank with error < 0.1; k = ceil(r n / m) when r n / m >= 2000,
 * else #{eig(K(X_m, X_m)) > 0.1 mu} on unscaled points; clipped to
 * [1, min(k_max, n)]).  m = 0 means min(n, 1000).
 */
afn_status afn_rank_estimate(const double *points, int64_t n, int32_t d, int32_t kernel, double l,
                             double mu, int32_t m, uint64_t seed, int32_t k_max, int64_t *k_out,
                             int64_t *r_out, int32_t *branch_out, void *stream);

/* ---- many systems: batched solves -------------------------------------- */

/* One independent system (K + mu I) a = b: the arguments of afn_build. */
typedef struct {
    const double *points;   /* n x d row-major FP64, host or device; read during the build */
    int64_t n;
    int32_t d;              /* 1..16 */
    int32_t kernel;         /* afn_kernel */
    double l, mu;           /* > 0 */
    int32_t k_max;          /* landmarks (clamped to [0, n]; Alg. 4 when opt.rank_mode = 1) */
    int32_t fsai_nnz;       /* w, nonzeros per row of G including the diagonal (1..128) */
} afn_system;

typedef struct afn_batch afn_batch;

typedef struct {
    int32_t converged;      /* columns whose FP64 relative residual reached tol */
    int32_t columns;        /* sum of nrhs */
    int32_t graph_launches; /* CUDA graph launches (opt.check_every iterations each) */
    int32_t iters_max;      /* largest per-column iteration count */
    double solve_ms;        /* device time of the whole solve */
    double group_ms;        /* host wall time until the grouped (mixed) systems finished */
    double single_ms;       /* host wall time until the last one-at-a-time (DF) system finished */
    int32_t single_systems; /* systems solved one at a time (precision other than MIXED) */
    int32_t pad_;
} afn_batch_solve_info;

/*
 * Builds the AFN preconditioners (Alg. 2, the factors of afn_build) of nsys
 * independent systems, several at a time on separate streams.  opt->precision
 * applies to every system as in afn_build (AFN_PREC_AUTO picks MIXED or DF per
 * system); mixed systems are later solved together, DF and FP64 ones one at
 * a time beside them.  opt->precond must be AFN_PRECOND_AFN (AFN_ERR_ARG
 * otherwise).  opt applies to every system (landmark policy,
 * rank mode, seed, max_iter, inner_tol = delta of the reliable updates,
 * check_every = PCG iterations per captured CUDA graph launch, stream for
 * the solves: NULL creates a private stream).  AFN_BUILD_THREADS in the
 * environment sets the number of building host threads (default 16).
 * Errors: those of afn_build, with the failing system's index in the
 * message; nothing is returned on failure.
 */
afn_status afn_build_batched(const afn_system *systems, int32_t nsys, const afn_options *opt,
                             afn_batch **out);

/*
 * Solves every system of the batch for its nrhs[s] right-hand sides.  The
 * mixed systems run the mixed-precision PCG of afn_solve (Alg. 5 with the
 * apply of Alg. 3; FP32 matvec/apply, FP64 scalars, FP64 residual
 * replacements; stop when the FP64 residual ||b - (K + mu I) x|| <= tol ||b||,
 * at most max_iter iterations a column), all advancing together: each step of
 * an iteration is one launch over the work of every mixed system that still
 * has an active column.  DF and FP64 systems are solved as by afn_solve, one
 * at a time on host threads, concurrently with the group.
 * rhs and x_out (host or device) hold the systems' n_s x nrhs[s] column-major
 * blocks one after the other, in original point order; iters and relres (host,
 * may be NULL) get sum(nrhs) entries in the same column order.  A system's
 * result does not depend on the other systems of the batch.
 * Returns AFN_ERR_NO_CONVERGE (x_out still written) when a column missed tol.
 */
afn_status afn_solve_batched(afn_batch *b, const double *rhs, const int32_t *nrhs, double tol,
                             double *x_out, int32_t *iters, double *relres,
                             afn_batch_solve_info *info);

/* build information of system `system` of the batch (as afn_get_build_info) */
afn_status afn_batch_build_info(const afn_batch *b, int32_t system, afn_build_info *info);
/* host wall time of afn_build_batched, ms */
double afn_batch_build_ms(const afn_batch *b);
void afn_batch_free(afn_batch *b);    /* NULL-safe */

/* ---- many systems: the serving loop ------------------------------------ */

typedef struct afn_server afn_server;

typedef struct {
    int64_t memory_budget;  /* device bytes for admitted requests; 0 = half the free memory */
    int32_t max_active;     /* admitted requests at once; 0 = no limit besides memory */
    int32_t build_threads;  /* host threads (each with a stream) building requests; 0 = 8 */
    afn_options opt;        /* build and solve options for every request; precond AFN;
                               precision AUTO by default (MIXED or DF per request) */
} afn_server_config;

typedef struct {
    int32_t status;         /* afn_status of the request */
    int32_t converged;      /* columns that reached tol */
    int32_t nrhs;
    int32_t pad_;
    double queue_ms;        /* submit -> admitted (memory reserved) */
    double build_ms;        /* preconditioner build (Alg. 2) on a build thread */
    double wait_ms;         /* built -> joined the running group */
    double solve_ms;        /* joined -> all columns stopped and result copied */
    double latency_ms;      /* submit -> done */
    int64_t device_bytes;   /* footprint reserved while admitted */
} afn_request_info;

typedef struct {
    int64_t submitted, completed, queued;
    int32_t active;         /* admitted, not finished */
    int32_t peak_live;      /* most requests advanced by one graph launch */
    int64_t graph_launches;
    int64_t reserved_bytes, peak_reserved_bytes, budget_bytes;
} afn_server_stats;

/* defaults: budget 0 (half the free memory), no count limit, 8 build
 * threads, afn_default_options with precision = AFN_PREC_AUTO */
void afn_server_default_config(afn_server_config *cfg);

/*
 * Starts a serving loop on the current device: one scheduler thread and
 * cfg->build_threads build threads.  Requests (afn_server_submit) are
 * admitted in arrival order while the sum of the admitted requests' device
 * footprints stays within the budget (a request larger than the budget runs
 * when nothing else is admitted); each is built (Alg. 2) on a build thread's
 * own stream; a mixed request then joins the group of running PCG solves
 * (the solve of afn_solve_batched, one launch per step for all requests) at
 * its next graph launch and leaves it when its columns have stopped, a DF or
 * FP64 request is solved on its build thread as by afn_solve; its device memory is
 * then released and its result kept in host memory until afn_server_result.
 * A request's solution is the same whatever other requests run beside it.
 * Errors: AFN_ERR_ARG (bad config), AFN_ERR_CUDA.
 */
afn_status afn_server_create(const afn_server_config *cfg, afn_server **out);

/* Queues one system (points n x d row-major, rhs n x nrhs column-major,
 * host or device; both are copied before the call returns).  *id identifies
 * the request.  Errors: AFN_ERR_ARG (bad sizes, NaN/Inf). */
afn_status afn_server_submit(afn_server *s, const afn_system *sys, const double *rhs,
                             int32_t nrhs, double tol, int64_t *id);

/* Up to max ids of finished requests (each reported once), waiting up to
 * wait_ms for the first one; *count = number written. */
afn_status afn_server_poll(afn_server *s, int64_t *ids, int32_t max, int32_t *count,
                           int32_t wait_ms);

/* Result of a finished request (x_out n x nrhs column-major, original point
 * order, host or device; iters/relres host, nrhs entries; any may be NULL),
 * then forgets the request.  Returns the request's status (AFN_ERR_BUSY when
 * it has not finished, AFN_ERR_ARG for an unknown id). */
afn_status afn_server_result(afn_server *s, int64_t id, double *x_out, int32_t *iters,
                             double *relres, afn_request_info *info);

afn_status afn_server_get_stats(afn_server *s, afn_server_stats *out);

/* Stops the loop (requests not yet finished are dropped) and releases
 * everything.  NULL-safe. */
void afn_server_destroy(afn_server *s);

#ifdef __cplusplus
}
#endif
#endif /* AFN_H */
