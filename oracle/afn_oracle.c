/*
 * afn_oracle.c -- plain, slow, FP64 CPU oracle for AFN-preconditioned CG
 * (Zhao, Xu, Huang, Chow, Xi: "An Adaptive Factorized Nystrom Preconditioner
 * for Regularized Kernel Matrices", arXiv 2304.05460).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may call, link or
 * load this file: only the test-suite, the smoke check and the benchmark's
 * CPU-baseline / reference arm use it.  It shares no code, header, table or
 * helper with the CUDA library; the two only meet through the seeded input
 * generators.
 *
 * Every function is a literal restatement of a definition or an algorithm of
 * the paper, in the paper's order, in double precision, with sequential sums
 * in ascending index order.  It is compiled with -ffp-contract=off so that no
 * multiply-add is fused and the results are the same on x86-64 and aarch64.
 * OpenMP is used only across independent rows (each row's arithmetic is
 * sequential), so results do not depend on the thread count.
 *
 * Layouts: every matrix is row-major.  Points are n x d row-major.
 * The FSAI factor G is stored ELL-style: row i has w slots, slot p holds the
 * column pattern[i*w+p] (or -1 for padding) and the value G[i*w+p]; the
 * diagonal entry (column i) is the last used slot of the row.
 *
 * Status codes returned by the functions: 0 ok, 1 bad argument,
 * 3 a matrix that must be SPD is not (a Cholesky pivot <= 0),
 * 4 PCG did not reach the tolerance within max_iter.
 *
 * The Nystrom preconditioner of Alg. 5's small-rank branch (Sec. 2, eq.
 * (nystrom1-smw)) is built literally in its orthonormal form, with a cyclic
 * Jacobi eigendecomposition; PCG takes either preconditioner.
 *
 * Parity: every function here is pinned by the CPU tests (closed forms,
 * brute force on tiny inputs, the paper's invariants); see the test files.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_GAUSSIAN 0
#define ORC_MATERN32 1

/* ------------------------------------------------------------------------ */
/* threads                                                                   */
/* ------------------------------------------------------------------------ */
void orc_set_threads(int t)
{
#ifdef _OPENMP
    if (t > 0) omp_set_num_threads(t);
#else
    (void)t;
#endif
}

int orc_get_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* Kernel functions: Gaussian, eq. (gaussianf) / Sec. 5 list; Matern-3/2,    */
/* Sec. 5 list.  r^2 is summed over t = 0..d-1 in ascending order.           */
/* ------------------------------------------------------------------------ */
double orc_sqdist(const double *x, const double *y, int d)
{
    double s = 0.0;
    for (int t = 0; t < d; ++t) {
        double u = x[t] - y[t];
        s = s + u * u;
    }
    return s;
}

double orc_kernel_from_sqdist(double r2, int kernel, double l)
{
    if (kernel == ORC_GAUSSIAN) {
        /* exp(-||x-y||^2 / l^2) */
        return exp(-(r2 / (l * l)));
    }
    /* (1 + sqrt(3) r / l) exp(-sqrt(3) r / l), r = ||x-y||_2 */
    double r = sqrt(r2);
    double t = sqrt(3.0) * r / l;
    return (1.0 + t) * exp(-t);
}

double orc_kernel_eval(const double *x, const double *y, int d, int kernel, double l)
{
    return orc_kernel_from_sqdist(orc_sqdist(x, y, d), kernel, l);
}

/* K[i*ny+j] = K(X_i, Y_j)  (the kernel matrix K_{X,Y} of Sec. 2) */
void orc_kernel_matrix(const double *X, int64_t nx, const double *Y, int64_t ny,
                       int d, int kernel, double l, double *K)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < nx; ++i)
        for (int64_t j = 0; j < ny; ++j)
            K[i * ny + j] = orc_kernel_eval(X + i * d, Y + j * d, d, kernel, l);
}

/* ------------------------------------------------------------------------ */
/* Matrix-free product y = (K + mu I) p for nrhs columns (eq. (Problem)).    */
/* p and y are n x nrhs column-major.  Row i sums j = 0..n-1 in order.       */
/* ------------------------------------------------------------------------ */
void orc_matvec(const double *X, int64_t n, int d, int kernel, double l, double mu,
                const double *p, int nrhs, double *y)
{
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < n; ++i) {
        for (int c = 0; c < nrhs; ++c) {
            double s = 0.0;
            const double *pc = p + (int64_t)c * n;
            for (int64_t j = 0; j < n; ++j)
                s = s + orc_kernel_eval(X + i * d, X + j * d, d, kernel, l) * pc[j];
            y[(int64_t)c * n + i] = s + mu * pc[i];
        }
    }
}

/* Same product with an explicit dense K (n x n row-major); identical sums. */
static void dense_matvec1(const double *K, int64_t n, double mu, const double *p, double *y)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        double s = 0.0;
        for (int64_t j = 0; j < n; ++j) s = s + K[i * n + j] * p[j];
        y[i] = s + mu * p[i];
    }
}

static void free_matvec1(const double *X, int64_t n, int d, int kernel, double l, double mu,
                         const double *p, double *y)
{
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < n; ++i) {
        double s = 0.0;
        for (int64_t j = 0; j < n; ++j)
            s = s + orc_kernel_eval(X + i * d, X + j * d, d, kernel, l) * p[j];
        y[i] = s + mu * p[i];
    }
}

/* ------------------------------------------------------------------------ */
/* Farthest point sampling, Algorithm 6 (Sec. 4.4) with the O(dkn) distance   */
/* vector.  Squared distances select the same argmax as distances.  Ties go  */
/* to the lowest index; an already selected point is excluded explicitly     */
/* (its entry is set to -1), so duplicated points are never chosen twice.    */
/* ------------------------------------------------------------------------ */
int orc_fps(const double *X, int64_t n, int d, int64_t k, int64_t start, int64_t *idx)
{
    if (k <= 0) return 0;
    if (k > n || start < 0 || start >= n) return 1;
    double *dm = (double *)malloc(sizeof(double) * (size_t)n);
    if (!dm) return 1;
    for (int64_t j = 0; j < n; ++j) dm[j] = INFINITY;
    idx[0] = start;
    dm[start] = -1.0;
    for (int64_t i = 1; i < k; ++i) {
        const double *xl = X + idx[i - 1] * d;
        for (int64_t j = 0; j < n; ++j) {
            if (dm[j] >= 0.0) {
                double r2 = orc_sqdist(X + j * d, xl, d);
                if (r2 < dm[j]) dm[j] = r2;
            }
        }
        int64_t best = -1;
        double bv = -INFINITY;
        for (int64_t j = 0; j < n; ++j)
            if (dm[j] > bv) { bv = dm[j]; best = j; }
        idx[i] = best;
        dm[best] = -1.0;
    }
    free(dm);
    return 0;
}

/* Alg. 6's start point: the point nearest the centroid (ties: lowest index).
 * The centroid sums each coordinate over j = 0..n-1 in order. */
int64_t orc_fps_centroid_start(const double *X, int64_t n, int d)
{
    double *c = (double *)calloc((size_t)d, sizeof(double));
    for (int t = 0; t < d; ++t) {
        double s = 0.0;
        for (int64_t j = 0; j < n; ++j) s = s + X[j * d + t];
        c[t] = s / (double)n;
    }
    int64_t best = 0;
    double bv = INFINITY;
    for (int64_t j = 0; j < n; ++j) {
        double r2 = orc_sqdist(X + j * d, c, d);
        if (r2 < bv) { bv = r2; best = j; }
    }
    free(c);
    return best;
}

/* ------------------------------------------------------------------------ */
/* Uniform sampling without replacement (Alg. 2 for d > 10; Alg. 4's         */
/* subsample): a partial Fisher-Yates shuffle of 0..n-1 driven by SplitMix64 */
/* (Steele, Lea, Flood, "Fast splittable pseudorandom number generators",    */
/* OOPSLA 2014).  idx[i] = the i-th drawn index.                             */
/* ------------------------------------------------------------------------ */
uint64_t orc_splitmix64_next(uint64_t *state)
{
    uint64_t z = (*state += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

int orc_uniform_sample(int64_t n, int64_t k, uint64_t seed, int64_t *idx)
{
    if (k < 0 || k > n) return 1;
    int64_t *a = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    for (int64_t j = 0; j < n; ++j) a[j] = j;
    uint64_t st = seed;
    for (int64_t i = 0; i < k; ++i) {
        uint64_t r = orc_splitmix64_next(&st);
        int64_t j = i + (int64_t)(r % (uint64_t)(n - i));
        int64_t t = a[i]; a[i] = a[j]; a[j] = t;
        idx[i] = a[i];
    }
    free(a);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Landmarks first (the 2x2 partition of Sec. 2): perm = [X_k in selection   */
/* order ; the other points in ascending original index].                    */
/* ------------------------------------------------------------------------ */
int orc_permutation(int64_t n, const int64_t *landmarks, int64_t k, int64_t *perm)
{
    char *used = (char *)calloc((size_t)(n > 0 ? n : 1), 1);
    for (int64_t i = 0; i < k; ++i) {
        if (landmarks[i] < 0 || landmarks[i] >= n || used[landmarks[i]]) { free(used); return 1; }
        used[landmarks[i]] = 1;
        perm[i] = landmarks[i];
    }
    int64_t p = k;
    for (int64_t j = 0; j < n; ++j)
        if (!used[j]) perm[p++] = j;
    free(used);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* FSAI sparsity pattern (Sec. 3.1): row i of X_r holds the w-1 nearest      */
/* points numbered less than i (ordered by (r^2, j) ascending) followed by i */
/* itself.  Rows with fewer than w-1 predecessors take all of them.           */
/* rowlen[i] = number of used slots; unused slots hold -1.                   */
/* ------------------------------------------------------------------------ */
/* One row of the pattern: the scan over j = 0..i-1 in ascending order with a
 * sorted candidate list of length m = min(i, w-1); bd/bj hold >= w-1 slots.
 * Returns the number of used slots (cnt + 1). */
static int32_t knn_row(const double *Xr, int d, int w, int64_t i, double *bd, int64_t *bj,
                       int32_t *prow)
{
    int64_t m = i < (int64_t)(w - 1) ? i : (int64_t)(w - 1);
    int64_t cnt = 0;
    for (int64_t j = 0; j < i && m > 0; ++j) {
        double r2 = orc_sqdist(Xr + i * d, Xr + j * d, d);
        /* candidates arrive in ascending j, so an equal distance never
         * displaces an entry already held (lower index wins ties) */
        if (cnt == m && !(r2 < bd[m - 1])) continue;
        int64_t pos = (cnt < m) ? cnt : m - 1;
        while (pos > 0 && r2 < bd[pos - 1]) {
            bd[pos] = bd[pos - 1];
            bj[pos] = bj[pos - 1];
            --pos;
        }
        bd[pos] = r2;
        bj[pos] = j;
        if (cnt < m) ++cnt;
    }
    for (int p = 0; p < w; ++p) prow[p] = -1;
    for (int64_t p = 0; p < cnt; ++p) prow[p] = (int32_t)bj[p];
    prow[cnt] = (int32_t)i;
    return (int32_t)(cnt + 1);
}

void orc_knn_pattern(const double *Xr, int64_t nr, int d, int w, int32_t *pat, int32_t *rowlen)
{
#pragma omp parallel
    {
        double *bd = (double *)malloc(sizeof(double) * (size_t)(w > 1 ? w : 1));
        int64_t *bj = (int64_t *)malloc(sizeof(int64_t) * (size_t)(w > 1 ? w : 1));
#pragma omp for schedule(dynamic, 8)
        for (int64_t i = 0; i < nr; ++i)
            rowlen[i] = knn_row(Xr, d, w, i, bd, bj, pat + i * w);
        free(bd);
        free(bj);
    }
}

/* The pattern rows rows[0..nrows) of the same definition (row i depends only
 * on points 0..i, so large problems are checked on a sample of rows at O(i d)
 * each).  pat: nrows x w. */
void orc_knn_rows(const double *Xr, int64_t nr, int d, int w, const int64_t *rows, int64_t nrows,
                  int32_t *pat)
{
    (void)nr;
#pragma omp parallel
    {
        double *bd = (double *)malloc(sizeof(double) * (size_t)(w > 1 ? w : 1));
        int64_t *bj = (int64_t *)malloc(sizeof(int64_t) * (size_t)(w > 1 ? w : 1));
#pragma omp for schedule(dynamic, 1)
        for (int64_t q = 0; q < nrows; ++q)
            (void)knn_row(Xr, d, w, rows[q], bd, bj, pat + q * w);
        free(bd);
        free(bj);
    }
}

/* ------------------------------------------------------------------------ */
/* Textbook Cholesky A = L L^T (Alg. 2, line "Perform Cholesky").  Column by */
/* column; the row loop below the pivot is independent per row.  Returns 0   */
/* or 3 (a pivot <= 0: A is not numerically SPD).                            */
/* ------------------------------------------------------------------------ */
int orc_cholesky(const double *A, int64_t k, double *L)
{
    memset(L, 0, sizeof(double) * (size_t)(k * k));
    for (int64_t j = 0; j < k; ++j) {
        double s = A[j * k + j];
        for (int64_t p = 0; p < j; ++p) s = s - L[j * k + p] * L[j * k + p];
        if (!(s > 0.0)) return 3;
        double ljj = sqrt(s);
        L[j * k + j] = ljj;
#pragma omp parallel for schedule(static) if (k - j > 256)
        for (int64_t i = j + 1; i < k; ++i) {
            double t = A[i * k + j];
            for (int64_t p = 0; p < j; ++p) t = t - L[i * k + p] * L[j * k + p];
            L[i * k + j] = t / ljj;
        }
    }
    return 0;
}

/* L x = b (forward substitution); L is k x k lower, row-major */
void orc_forward(const double *L, int64_t k, const double *b, double *x)
{
    for (int64_t i = 0; i < k; ++i) {
        double s = b[i];
        for (int64_t p = 0; p < i; ++p) s = s - L[i * k + p] * x[p];
        x[i] = s / L[i * k + i];
    }
}

/* L^T x = b (backward substitution) */
void orc_backward(const double *L, int64_t k, const double *b, double *x)
{
    for (int64_t i = k - 1; i >= 0; --i) {
        double s = b[i];
        for (int64_t p = i + 1; p < k; ++p) s = s - L[p * k + i] * x[p];
        x[i] = s / L[i * k + i];
    }
}

/* ------------------------------------------------------------------------ */
/* One FSAI row, Alg. 1: G_{i,s} = e_w^T A^{-1} / sqrt(e_w^T A^{-1} e_w)     */
/* with A the pattern block (w_i x w_i, row-major).  A y = e_w is solved by  */
/* a Cholesky factorisation and two triangular solves.  Returns 0 or 3.       */
/* ------------------------------------------------------------------------ */
int orc_fsai_row(const double *A, int m, double *g)
{
    double *R = (double *)malloc(sizeof(double) * (size_t)(m * m));
    double *e = (double *)calloc((size_t)m, sizeof(double));
    double *z = (double *)malloc(sizeof(double) * (size_t)m);
    int st = orc_cholesky(A, m, R);
    if (st == 0) {
        e[m - 1] = 1.0;
        orc_forward(R, m, e, z);
        orc_backward(R, m, z, g);            /* g = y = A^{-1} e_w */
        double yw = g[m - 1];
        if (!(yw > 0.0)) st = 3;
        else {
            double sc = sqrt(yw);
            for (int p = 0; p < m; ++p) g[p] = g[p] / sc;
        }
    }
    free(R); free(e); free(z);
    return st;
}

/* ------------------------------------------------------------------------ */
/* AFN construction, Alg. 2, given the landmark indices (FPS or uniform):    */
/*   perm = [X_k ; X_r];  L = chol(K11 + mu I);  K12 = K(X_k, X_r);          */
/*   G = FSAI of S = K22 + mu I - K12^T (K11 + mu I)^{-1} K12 (Sec. 3.1-3.2) */
/* The pattern block of S for each row is formed literally: each pattern     */
/* column c of K12 gets two triangular solves v_c = L^{-T} L^{-1} K12[:,c],  */
/* and A_ab = K(x_a, x_b) + mu [a==b] - K12[:,a]^T v_b.                      */
/* Outputs: perm[n]; L[k*k]; K12[k*nr]; pat[nr*w]; rowlen[nr]; G[nr*w].      */
/* Returns 0, 1 (argument), 3 (K11+mu I or a pattern block not SPD).         */
/* ------------------------------------------------------------------------ */
int orc_afn_build(const double *X, int64_t n, int d, int kernel, double l, double mu,
                  int64_t k, int w, const int64_t *landmarks,
                  int64_t *perm, double *L, double *K12, int32_t *pat, int32_t *rowlen, double *G)
{
    if (n < 1 || d < 1 || !(l > 0) || !(mu > 0) || k < 0 || k > n || w < 1) return 1;
    int64_t nr = n - k;
    if (orc_permutation(n, landmarks, k, perm)) return 1;
    double *Xp = (double *)malloc(sizeof(double) * (size_t)(n * d));
    for (int64_t i = 0; i < n; ++i)
        for (int t = 0; t < d; ++t) Xp[i * d + t] = X[perm[i] * d + t];
    const double *Xk = Xp, *Xr = Xp + k * d;
    int st = 0;
    if (k > 0) {
        double *A11 = (double *)malloc(sizeof(double) * (size_t)(k * k));
        orc_kernel_matrix(Xk, k, Xk, k, d, kernel, l, A11);
        for (int64_t i = 0; i < k; ++i) A11[i * k + i] = A11[i * k + i] + mu;
        st = orc_cholesky(A11, k, L);
        free(A11);
        if (st) { free(Xp); return st; }
        orc_kernel_matrix(Xk, k, Xr, nr, d, kernel, l, K12);
    }
    if (nr == 0) { free(Xp); return 0; }
    orc_knn_pattern(Xr, nr, d, w, pat, rowlen);
    int bad = 0;
#pragma omp parallel
    {
        double *V = (double *)malloc(sizeof(double) * (size_t)((k > 0 ? k : 1) * w));
        double *col = (double *)malloc(sizeof(double) * (size_t)(k > 0 ? k : 1));
        double *tmp = (double *)malloc(sizeof(double) * (size_t)(k > 0 ? k : 1));
        double *A = (double *)malloc(sizeof(double) * (size_t)(w * w));
        double *g = (double *)malloc(sizeof(double) * (size_t)w);
#pragma omp for schedule(dynamic, 4)
        for (int64_t i = 0; i < nr; ++i) {
            int m = rowlen[i];
            const int32_t *s = pat + i * w;
            /* v_c = (K11 + mu I)^{-1} K12[:, s_c] by two triangular solves */
            for (int c = 0; c < m && k > 0; ++c) {
                for (int64_t t = 0; t < k; ++t) col[t] = K12[t * nr + s[c]];
                orc_forward(L, k, col, tmp);
                orc_backward(L, k, tmp, V + (int64_t)c * k);
            }
            for (int a = 0; a < m; ++a) {
                for (int b = 0; b < m; ++b) {
                    double v = orc_kernel_eval(Xr + (int64_t)s[a] * d, Xr + (int64_t)s[b] * d, d, kernel, l);
                    if (a == b) v = v + mu;
                    double q = 0.0;
                    for (int64_t t = 0; t < k; ++t) q = q + K12[t * nr + s[a]] * V[(int64_t)b * k + t];
                    A[a * m + b] = v - q;
                }
            }
            for (int p = 0; p < w; ++p) G[i * w + p] = 0.0;
            int rs = orc_fsai_row(A, m, g);
            if (rs) {
#pragma omp atomic write
                bad = rs;
            } else {
                for (int p = 0; p < m; ++p) G[i * w + p] = g[p];
            }
        }
        free(V); free(col); free(tmp); free(A); free(g);
    }
    free(Xp);
    return bad;
}

/* ------------------------------------------------------------------------ */
/* AFN apply, Alg. 3 (vectors in permuted order, length n = k + nr):          */
/*   z  = L^{-T} L^{-1} r1                                                   */
/*   s2 = G^T G (r2 - K12^T z)                                               */
/*   s1 = L^{-T} L^{-1} (r1 - K12 s2)                                        */
/* G^T y is a scatter over the rows of G in ascending row order.             */
/* ------------------------------------------------------------------------ */
void orc_afn_apply(int64_t k, int64_t nr, int w, const double *L, const double *K12,
                   const int32_t *pat, const double *G, const double *r, double *s)
{
    const double *r1 = r, *r2 = r + k;
    double *s1 = s, *s2 = s + k;
    double *tmp = (double *)malloc(sizeof(double) * (size_t)(k > 0 ? k : 1));
    double *z = (double *)malloc(sizeof(double) * (size_t)(k > 0 ? k : 1));
    double *t = (double *)malloc(sizeof(double) * (size_t)(nr > 0 ? nr : 1));
    double *y = (double *)malloc(sizeof(double) * (size_t)(nr > 0 ? nr : 1));
    if (k > 0) {
        orc_forward(L, k, r1, tmp);
        orc_backward(L, k, tmp, z);
    }
    for (int64_t j = 0; j < nr; ++j) {
        double q = 0.0;
        for (int64_t i = 0; i < k; ++i) q = q + K12[i * nr + j] * z[i];
        t[j] = r2[j] - q;
    }
    for (int64_t i = 0; i < nr; ++i) {
        double q = 0.0;
        for (int p = 0; p < w; ++p) {
            int32_t c = pat[i * w + p];
            if (c >= 0) q = q + G[i * w + p] * t[c];
        }
        y[i] = q;
    }
    for (int64_t j = 0; j < nr; ++j) s2[j] = 0.0;
    for (int64_t i = 0; i < nr; ++i)
        for (int p = 0; p < w; ++p) {
            int32_t c = pat[i * w + p];
            if (c >= 0) s2[c] = s2[c] + G[i * w + p] * y[i];
        }
    if (k > 0) {
        for (int64_t i = 0; i < k; ++i) {
            double q = 0.0;
            for (int64_t j = 0; j < nr; ++j) q = q + K12[i * nr + j] * s2[j];
            z[i] = r1[i] - q;
        }
        orc_forward(L, k, z, tmp);
        orc_backward(L, k, tmp, s1);
    }
    free(tmp); free(z); free(t); free(y);
}

/* ------------------------------------------------------------------------ */
/* Dense preconditioner M, two ways, for tiny n (n x n row-major, permuted   */
/* order).  (a) eq. (factorized-form): M = F F^T with                       */
/*     F = [ L , 0 ; K12^T L^{-T} , G^{-1} ].                                */
/* (b) eq. (realM): M = [ K11+mu I , K12 ; K12^T ,                           */
/*                        (G^T G)^{-1} + K12^T (K11+mu I)^{-1} K12 ].        */
/* G^{-1} is formed column by column by forward substitution with dense G.  */
/* ------------------------------------------------------------------------ */
static double *dense_G(int64_t nr, int w, const int32_t *pat, const double *G)
{
    double *D = (double *)calloc((size_t)(nr * nr > 0 ? nr * nr : 1), sizeof(double));
    for (int64_t i = 0; i < nr; ++i)
        for (int p = 0; p < w; ++p)
            if (pat[i * w + p] >= 0) D[i * nr + pat[i * w + p]] = G[i * w + p];
    return D;
}

static double *lower_inverse(const double *T, int64_t m)
{
    double *Inv = (double *)calloc((size_t)(m * m > 0 ? m * m : 1), sizeof(double));
    double *e = (double *)calloc((size_t)(m > 0 ? m : 1), sizeof(double));
    double *x = (double *)malloc(sizeof(double) * (size_t)(m > 0 ? m : 1));
    for (int64_t c = 0; c < m; ++c) {
        memset(e, 0, sizeof(double) * (size_t)m);
        e[c] = 1.0;
        orc_forward(T, m, e, x);
        for (int64_t i = 0; i < m; ++i) Inv[i * m + c] = x[i];
    }
    free(e); free(x);
    return Inv;
}

void orc_dense_M_factored(int64_t k, int64_t nr, int w, const double *L, const double *K12,
                          const int32_t *pat, const double *G, double *M)
{
    int64_t n = k + nr;
    double *F = (double *)calloc((size_t)(n * n), sizeof(double));
    for (int64_t i = 0; i < k; ++i)
        for (int64_t j = 0; j <= i; ++j) F[i * n + j] = L[i * k + j];
    /* (K12^T L^{-T})_{j,:} = (L^{-1} K12[:, j])^T */
    double *tmp = (double *)malloc(sizeof(double) * (size_t)(k > 0 ? k : 1));
    double *col = (double *)malloc(sizeof(double) * (size_t)(k > 0 ? k : 1));
    for (int64_t j = 0; j < nr && k > 0; ++j) {
        for (int64_t t = 0; t < k; ++t) col[t] = K12[t * nr + j];
        orc_forward(L, k, col, tmp);
        for (int64_t t = 0; t < k; ++t) F[(k + j) * n + t] = tmp[t];
    }
    double *Gd = dense_G(nr, w, pat, G);
    double *Gi = lower_inverse(Gd, nr);
    for (int64_t i = 0; i < nr; ++i)
        for (int64_t j = 0; j < nr; ++j) F[(k + i) * n + k + j] = Gi[i * nr + j];
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = 0; j < n; ++j) {
            double s = 0.0;
            for (int64_t t = 0; t < n; ++t) s = s + F[i * n + t] * F[j * n + t];
            M[i * n + j] = s;
        }
    free(F); free(tmp); free(col); free(Gd); free(Gi);
}

void orc_dense_M_expanded(const double *Xp, int64_t n, int d, int kernel, double l, double mu,
                          int64_t k, int w, const double *L, const double *K12,
                          const int32_t *pat, const double *G, double *M)
{
    int64_t nr = n - k;
    for (int64_t i = 0; i < k; ++i)
        for (int64_t j = 0; j < k; ++j)
            M[i * n + j] = orc_kernel_eval(Xp + i * d, Xp + j * d, d, kernel, l) + (i == j ? mu : 0.0);
    for (int64_t i = 0; i < k; ++i)
        for (int64_t j = 0; j < nr; ++j) {
            M[i * n + k + j] = K12[i * nr + j];
            M[(k + j) * n + i] = K12[i * nr + j];
        }
    /* (G^T G)^{-1} = G^{-1} G^{-T} */
    double *Gd = dense_G(nr, w, pat, G);
    double *Gi = lower_inverse(Gd, nr);
    /* V = (K11 + mu I)^{-1} K12 column by column */
    double *V = (double *)malloc(sizeof(double) * (size_t)((k > 0 ? k : 1) * (nr > 0 ? nr : 1)));
    double *tmp = (double *)malloc(sizeof(double) * (size_t)(k > 0 ? k : 1));
    double *col = (double *)malloc(sizeof(double) * (size_t)(k > 0 ? k : 1));
    for (int64_t j = 0; j < nr && k > 0; ++j) {
        for (int64_t t = 0; t < k; ++t) col[t] = K12[t * nr + j];
        orc_forward(L, k, col, tmp);
        orc_backward(L, k, tmp, col);
        for (int64_t t = 0; t < k; ++t) V[t * nr + j] = col[t];
    }
    for (int64_t a = 0; a < nr; ++a)
        for (int64_t b = 0; b < nr; ++b) {
            double s = 0.0;
            for (int64_t t = 0; t < nr; ++t) s = s + Gi[a * nr + t] * Gi[b * nr + t];
            double q = 0.0;
            for (int64_t t = 0; t < k; ++t) q = q + K12[t * nr + a] * V[t * nr + b];
            M[(k + a) * n + k + b] = s + q;
        }
    free(Gd); free(Gi); free(V); free(tmp); free(col);
}

/* ------------------------------------------------------------------------ */
/* Preconditioned conjugate gradient (Alg. 5, line "Solve ... using PCG"),   */
/* textbook Hestenes-Stiefel recurrences, one right-hand side, x0 = 0,       */
/* stop when the recursive ||r||_2 <= tol ||b||_2 (Sec. 5: relative residual */
/* norm).  The true residual b - (K + mu I) x is then recomputed; if it is   */
/* above tol, PCG restarts from x (at most max_restarts times), all          */
/* iterations counted.  Xp is the permuted point set (the preconditioner's   */
/* order); with L == NULL and G == NULL the preconditioner is the identity   */
/* (plain CG).  iters = number of products with K + mu I inside the loops.   */
/* Returns 0, or 4 when max_iter is reached first.                           */
/* ------------------------------------------------------------------------ */
/* the preconditioner of one PCG run: s = M^{-1} r (identity when apply is NULL) */
typedef struct {
    void (*apply)(const void *ctx, const double *r, double *s);
    const void *ctx;
} precond_t;

typedef struct {
    int64_t k, nr;
    int w;
    const double *L, *K12, *G;
    const int32_t *pat;
} afn_ctx_t;

static void afn_apply_cb(const void *c, const double *r, double *s)
{
    const afn_ctx_t *a = (const afn_ctx_t *)c;
    orc_afn_apply(a->k, a->nr, a->w, a->L, a->K12, a->pat, a->G, r, s);
}

static int pcg_core(const double *Xp, int64_t n, int d, int kernel, double l, double mu,
                    precond_t pc, const double *b, double tol, int max_iter, int max_restarts,
                    double *x, int *iters, double *relres)
{
    int ident = (pc.apply == NULL);
    double *Kd = NULL;
    if (n <= 4096) {
        Kd = (double *)malloc(sizeof(double) * (size_t)(n * n));
        orc_kernel_matrix(Xp, n, Xp, n, d, kernel, l, Kd);
    }
    double *r = (double *)malloc(sizeof(double) * (size_t)n);
    double *z = (double *)malloc(sizeof(double) * (size_t)n);
    double *p = (double *)malloc(sizeof(double) * (size_t)n);
    double *q = (double *)malloc(sizeof(double) * (size_t)n);
    double bn = 0.0;
    for (int64_t i = 0; i < n; ++i) bn = bn + b[i] * b[i];
    bn = sqrt(bn);
    for (int64_t i = 0; i < n; ++i) x[i] = 0.0;
    int it = 0, status = 4;
    double rel = 1.0;
    if (bn == 0.0) { status = 0; rel = 0.0; }
    for (int restart = 0; restart <= max_restarts && status != 0; ++restart) {
        /* r = b - (K + mu I) x */
        if (Kd) dense_matvec1(Kd, n, mu, x, q); else free_matvec1(Xp, n, d, kernel, l, mu, x, q);
        for (int64_t i = 0; i < n; ++i) r[i] = b[i] - q[i];
        if (ident) memcpy(z, r, sizeof(double) * (size_t)n);
        else pc.apply(pc.ctx, r, z);
        memcpy(p, z, sizeof(double) * (size_t)n);
        double rho = 0.0;
        for (int64_t i = 0; i < n; ++i) rho = rho + r[i] * z[i];
        int conv = 0;
        while (it < max_iter) {
            if (Kd) dense_matvec1(Kd, n, mu, p, q); else free_matvec1(Xp, n, d, kernel, l, mu, p, q);
            ++it;
            double pq = 0.0;
            for (int64_t i = 0; i < n; ++i) pq = pq + p[i] * q[i];
            double alpha = rho / pq;
            for (int64_t i = 0; i < n; ++i) x[i] = x[i] + alpha * p[i];
            for (int64_t i = 0; i < n; ++i) r[i] = r[i] - alpha * q[i];
            double rn = 0.0;
            for (int64_t i = 0; i < n; ++i) rn = rn + r[i] * r[i];
            if (sqrt(rn) <= tol * bn) { conv = 1; break; }
            if (ident) memcpy(z, r, sizeof(double) * (size_t)n);
            else pc.apply(pc.ctx, r, z);
            double rho1 = 0.0;
            for (int64_t i = 0; i < n; ++i) rho1 = rho1 + r[i] * z[i];
            double beta = rho1 / rho;
            for (int64_t i = 0; i < n; ++i) p[i] = z[i] + beta * p[i];
            rho = rho1;
        }
        /* true residual */
        if (Kd) dense_matvec1(Kd, n, mu, x, q); else free_matvec1(Xp, n, d, kernel, l, mu, x, q);
        double tn = 0.0;
        for (int64_t i = 0; i < n; ++i) { double u = b[i] - q[i]; tn = tn + u * u; }
        rel = sqrt(tn) / bn;
        if (conv && rel <= tol) status = 0;
        if (!conv) break;
    }
    *iters = it;
    *relres = rel;
    free(Kd); free(r); free(z); free(p); free(q);
    return status;
}

/* PCG with the AFN preconditioner (L == NULL and G == NULL: plain CG) */
int orc_pcg(const double *Xp, int64_t n, int d, int kernel, double l, double mu,
            int64_t k, int w, const double *L, const double *K12, const int32_t *pat,
            const double *G, const double *b, double tol, int max_iter, int max_restarts,
            double *x, int *iters, double *relres)
{
    afn_ctx_t a = {k, n - k, w, L, K12, G, pat};
    precond_t pc = {NULL, NULL};
    if (!(L == NULL && G == NULL)) { pc.apply = afn_apply_cb; pc.ctx = &a; }
    return pcg_core(Xp, n, d, kernel, l, mu, pc, b, tol, max_iter, max_restarts, x, iters, relres);
}

/* ------------------------------------------------------------------------ */
/* Cyclic Jacobi eigendecomposition of a symmetric m x m matrix (Golub &     */
/* Van Loan, Matrix Computations, Alg. 8.5.3 with the symmetric Schur        */
/* rotation of Alg. 8.5.1): A (row-major, overwritten) -> eigenvalues w[m]  */
/* and eigenvectors as the columns of V (row-major m x m).  Sweeps until    */
/* off(A) <= 1e-15 ||A||_F (at most 60 sweeps).                              */
/* ------------------------------------------------------------------------ */
void orc_jacobi_eig(double *A, int64_t m, double *V, double *w)
{
    for (int64_t i = 0; i < m; ++i)
        for (int64_t j = 0; j < m; ++j) V[i * m + j] = (i == j) ? 1.0 : 0.0;
    double fro = 0.0;
    for (int64_t i = 0; i < m * m; ++i) fro = fro + A[i] * A[i];
    fro = sqrt(fro);
    for (int sweep = 0; sweep < 60; ++sweep) {
        double off = 0.0;
        for (int64_t p = 0; p < m; ++p)
            for (int64_t q = p + 1; q < m; ++q) off = off + 2.0 * A[p * m + q] * A[p * m + q];
        if (sqrt(off) <= 1e-15 * fro) break;
        for (int64_t p = 0; p < m - 1; ++p)
            for (int64_t q = p + 1; q < m; ++q) {
                double apq = A[p * m + q];
                if (apq == 0.0) continue;
                /* symmetric Schur: c, s annihilating A[p][q] */
                double tau = (A[q * m + q] - A[p * m + p]) / (2.0 * apq);
                double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                double c = 1.0 / sqrt(1.0 + t * t), sn = t * c;
                /* A <- J^T A J with J the rotation in the (p, q) plane */
                for (int64_t i = 0; i < m; ++i) {
                    double aip = A[i * m + p], aiq = A[i * m + q];
                    A[i * m + p] = c * aip - sn * aiq;
                    A[i * m + q] = sn * aip + c * aiq;
                }
                for (int64_t j = 0; j < m; ++j) {
                    double apj = A[p * m + j], aqj = A[q * m + j];
                    A[p * m + j] = c * apj - sn * aqj;
                    A[q * m + j] = sn * apj + c * aqj;
                }
                for (int64_t i = 0; i < m; ++i) {
                    double vip = V[i * m + p], viq = V[i * m + q];
                    V[i * m + p] = c * vip - sn * viq;
                    V[i * m + q] = sn * vip + c * viq;
                }
            }
    }
    for (int64_t i = 0; i < m; ++i) w[i] = A[i * m + i];
}

/* ------------------------------------------------------------------------ */
/* Column-sampling Nystrom preconditioner (Sec. 2, eq. (sampling-based-     */
/* nystrom)) in the orthonormal form of eq. (nystrom1-smw).                  */
/* Reading: K_nys = Y K_SS^+ Y^T with Y = K(X, X_S) (n x k) is formed as      */
/* B B^T, B = Y L^{-T}, L = chol(K_SS + nu I), nu = n 2^-52 (the shift makes */
/* the pseudoinverse of a numerically singular K_SS a Cholesky factor); the  */
/* thin SVD B = U Sigma V^T comes from the eigendecomposition of B^T B       */
/* (Jacobi above): Lambda = Sigma^2, U = B V Sigma^{-1}, keeping the         */
/* eigenpairs with sigma^2 > 1e-14 max sigma^2 (rank r <= k).               */
/* Xp: points in the permuted order, landmarks first.  U: n x k row-major   */
/* (first r columns used), lam[k].  Returns 0, or 3 if K_SS + nu I is not    */
/* positive definite.                                                         */
/* ------------------------------------------------------------------------ */
int orc_nystrom_build(const double *Xp, int64_t n, int d, int kernel, double l, int64_t k,
                      double *U, double *lam, int64_t *rank)
{
    *rank = 0;
    if (k == 0) return 0;
    const double nu = (double)n * ldexp(1.0, -52);
    double *A = (double *)malloc(sizeof(double) * (size_t)(k * k));
    double *L = (double *)malloc(sizeof(double) * (size_t)(k * k));
    orc_kernel_matrix(Xp, k, Xp, k, d, kernel, l, A);
    for (int64_t i = 0; i < k; ++i) A[i * k + i] = A[i * k + i] + nu;
    int st = orc_cholesky(A, k, L);
    if (st) { free(A); free(L); return st; }
    /* B (n x k): row i = L^{-1} K(X_S, x_i), by forward substitution */
    double *B = (double *)malloc(sizeof(double) * (size_t)(n * k));
#pragma omp parallel
    {
        double *col = (double *)malloc(sizeof(double) * (size_t)k);
#pragma omp for
        for (int64_t i = 0; i < n; ++i) {
            for (int64_t t = 0; t < k; ++t)
                col[t] = orc_kernel_eval(Xp + t * d, Xp + i * d, d, kernel, l);
            orc_forward(L, k, col, B + i * k);
        }
        free(col);
    }
    /* B^T B (k x k), then its eigendecomposition */
    for (int64_t a = 0; a < k; ++a)
        for (int64_t c = 0; c < k; ++c) {
            double v = 0.0;
            for (int64_t i = 0; i < n; ++i) v = v + B[i * k + a] * B[i * k + c];
            A[a * k + c] = v;
        }
    double *V = (double *)malloc(sizeof(double) * (size_t)(k * k));
    double *w = (double *)malloc(sizeof(double) * (size_t)k);
    orc_jacobi_eig(A, k, V, w);
    double wmax = 0.0;
    for (int64_t j = 0; j < k; ++j) wmax = fmax(wmax, w[j]);
    int64_t r = 0;
    for (int64_t j = 0; j < k; ++j) {
        if (!(w[j] > 1e-14 * wmax)) continue;
        /* column r of U = B v_j / sigma_j */
        double sig = sqrt(w[j]);
        for (int64_t i = 0; i < n; ++i) {
            double v = 0.0;
            for (int64_t t = 0; t < k; ++t) v = v + B[i * k + t] * V[t * k + j];
            U[i * k + r] = v / sig;
        }
        lam[r] = w[j];
        ++r;
    }
    *rank = r;
    free(A); free(L); free(B); free(V); free(w);
    return 0;
}

/* eq. (nystrom1-smw): s = U (Lambda + mu I)^{-1} U^T r + (r - U U^T r) / mu  */
void orc_nystrom_apply(int64_t n, int64_t k, int64_t r, const double *U, const double *lam,
                       double mu, const double *rin, double *s)
{
    double *y = (double *)malloc(sizeof(double) * (size_t)(r > 0 ? r : 1));
    for (int64_t j = 0; j < r; ++j) {
        double v = 0.0;
        for (int64_t i = 0; i < n; ++i) v = v + U[i * k + j] * rin[i];
        y[j] = v;
    }
    for (int64_t i = 0; i < n; ++i) {
        double a = 0.0, b = 0.0;
        for (int64_t j = 0; j < r; ++j) {
            a = a + U[i * k + j] * (y[j] / (lam[j] + mu));
            b = b + U[i * k + j] * y[j];
        }
        s[i] = a + (rin[i] - b) / mu;
    }
    free(y);
}

typedef struct {
    int64_t n, k, r;
    const double *U, *lam;
    double mu;
} nys_ctx_t;

static void nys_apply_cb(const void *c, const double *r, double *s)
{
    const nys_ctx_t *a = (const nys_ctx_t *)c;
    orc_nystrom_apply(a->n, a->k, a->r, a->U, a->lam, a->mu, r, s);
}

/* PCG with the Nystrom preconditioner (Alg. 5, the k < 2000 branch) */
int orc_pcg_nystrom(const double *Xp, int64_t n, int d, int kernel, double l, double mu,
                    int64_t k, int64_t r, const double *U, const double *lam, const double *b,
                    double tol, int max_iter, int max_restarts, double *x, int *iters,
                    double *relres)
{
    nys_ctx_t a = {n, k, r, U, lam, mu};
    precond_t pc = {nys_apply_cb, &a};
    return pcg_core(Xp, n, d, kernel, l, mu, pc, b, tol, max_iter, max_restarts, x, iters, relres);
}

/* Direct solve (K + mu I) x = b by a dense Cholesky factorisation, for the
 * plain result a* = (K + mu I)^{-1} b (eq. (Problem)); nrhs columns,
 * column-major.  Returns 0 or 3. */
int orc_dense_solve(const double *X, int64_t n, int d, int kernel, double l, double mu,
                    const double *b, int nrhs, double *x)
{
    double *A = (double *)malloc(sizeof(double) * (size_t)(n * n));
    double *C = (double *)malloc(sizeof(double) * (size_t)(n * n));
    double *t = (double *)malloc(sizeof(double) * (size_t)n);
    orc_kernel_matrix(X, n, X, n, d, kernel, l, A);
    for (int64_t i = 0; i < n; ++i) A[i * n + i] = A[i * n + i] + mu;
    int st = orc_cholesky(A, n, C);
    if (st == 0)
        for (int c = 0; c < nrhs; ++c) {
            orc_forward(C, n, b + (int64_t)c * n, t);
            orc_backward(C, n, t, x + (int64_t)c * n);
        }
    free(A); free(C); free(t);
    return st;
}

/* ------------------------------------------------------------------------ */
/* Symmetric eigenvalue tools for Alg. 4: Householder tridiagonalisation     */
/* (Golub & Van Loan, Matrix Computations, Alg. 8.3.1) and the Sturm-sequence */
/* count of eigenvalues below a shift (Golub & Van Loan Sec. 8.4.1).          */
/* A is m x m row-major, symmetric, overwritten.  dg[m], of[m-1] out.        */
/* ------------------------------------------------------------------------ */
void orc_tridiagonalize(double *A, int64_t m, double *dg, double *of)
{
    double *v = (double *)malloc(sizeof(double) * (size_t)(m > 0 ? m : 1));
    double *p = (double *)malloc(sizeof(double) * (size_t)(m > 0 ? m : 1));
    for (int64_t j = 0; j + 2 < m; ++j) {
        int64_t len = m - j - 1;
        double nx = 0.0;
        for (int64_t i = 0; i < len; ++i) nx = nx + A[(j + 1 + i) * m + j] * A[(j + 1 + i) * m + j];
        nx = sqrt(nx);
        double x0 = A[(j + 1) * m + j];
        dg[j] = A[j * m + j];
        if (nx == 0.0) { of[j] = 0.0; continue; }
        double alpha = (x0 >= 0.0) ? -nx : nx;          /* H x = alpha e1 */
        for (int64_t i = 0; i < len; ++i) v[i] = A[(j + 1 + i) * m + j];
        v[0] = v[0] - alpha;
        double vv = 0.0;
        for (int64_t i = 0; i < len; ++i) vv = vv + v[i] * v[i];
        of[j] = alpha;
        if (vv == 0.0) continue;
        double beta = 2.0 / vv;
        /* p = beta A22 v ; w = p - (beta/2)(p^T v) v ; A22 -= v w^T + w v^T */
#pragma omp parallel for schedule(static) if (len > 256)
        for (int64_t a = 0; a < len; ++a) {
            double s = 0.0;
            for (int64_t b = 0; b < len; ++b) s = s + A[(j + 1 + a) * m + j + 1 + b] * v[b];
            p[a] = beta * s;
        }
        double pv = 0.0;
        for (int64_t a = 0; a < len; ++a) pv = pv + p[a] * v[a];
        double kk = 0.5 * beta * pv;
        for (int64_t a = 0; a < len; ++a) p[a] = p[a] - kk * v[a];
#pragma omp parallel for schedule(static) if (len > 256)
        for (int64_t a = 0; a < len; ++a)
            for (int64_t b = 0; b < len; ++b)
                A[(j + 1 + a) * m + j + 1 + b] = A[(j + 1 + a) * m + j + 1 + b] - v[a] * p[b] - p[a] * v[b];
    }
    if (m >= 2) {
        dg[m - 2] = A[(m - 2) * m + m - 2];
        of[m - 2] = A[(m - 1) * m + m - 2];
    }
    if (m >= 1) dg[m - 1] = A[(m - 1) * m + m - 1];
    free(v); free(p);
}

/* number of eigenvalues of the symmetric tridiagonal (dg, of) below sigma */
int64_t orc_sturm_count(const double *dg, const double *of, int64_t m, double sigma)
{
    int64_t cnt = 0;
    double q = 1.0;
    for (int64_t i = 0; i < m; ++i) {
        double e2 = (i > 0) ? of[i - 1] * of[i - 1] : 0.0;
        q = (dg[i] - sigma) - (i > 0 ? e2 / q : 0.0);
        if (q == 0.0) q = -1e-300;   /* a zero pivot counts as just below */
        if (q < 0.0) ++cnt;
    }
    return cnt;
}

/* largest eigenvalue of the tridiagonal by bisection on the Sturm count */
double orc_tridiag_max_eig(const double *dg, const double *of, int64_t m)
{
    double lo = INFINITY, hi = -INFINITY;
    for (int64_t i = 0; i < m; ++i) {
        double rad = (i > 0 ? fabs(of[i - 1]) : 0.0) + (i + 1 < m ? fabs(of[i]) : 0.0);
        if (dg[i] - rad < lo) lo = dg[i] - rad;
        if (dg[i] + rad > hi) hi = dg[i] + rad;
    }
    for (int it = 0; it < 200; ++it) {
        double mid = 0.5 * (lo + hi);
        if (!(mid > lo && mid < hi)) break;
        if (orc_sturm_count(dg, of, m, mid) == m) hi = mid; else lo = mid;
    }
    return 0.5 * (lo + hi);
}

/* ------------------------------------------------------------------------ */
/* Nystrom rank estimation, Alg. 4, with these readings of the unspecified   */
/* parts: the subsample is the first m draws of the uniform sampler above;    */
/* FPS on the scaled subsample starts at its index 0; the Nystrom error of   */
/* rank r is ||E_r||_2 / ||K_m||_2 with E_r the Schur complement of K_m (in  */
/* FPS order) after its first r pivots (a pivot <= m * 2^-52 * max diag is   */
/* treated as zero, i.e. that point is already in the span); r is the       */
/* smallest rank with error < 0.1 (found by bisection over r, valid because  */
/* E_{r+1} is a Schur complement of E_r, so its 2-norm cannot grow);         */
/* k = ceil(r n / m); the branch test of Alg. 4 is r n / m >= 2000; below it */
/* k = #{eigenvalues of K(X_m, X_m), unscaled points, > 0.1 mu}; finally k   */
/* is clipped to [1, min(k_max, n)].                                         */
/* r_out (may be NULL) receives r; branch_out receives 0 (rn/m) or 1 (eig).  */
/* ------------------------------------------------------------------------ */
static int nys_error_below(const double *Ko, const double *Lo, int64_t m, int64_t r, double theta)
{
    int64_t s = m - r;
    if (s <= 0) return 1;
    double *E = (double *)malloc(sizeof(double) * (size_t)(s * s));
    double *dg = (double *)malloc(sizeof(double) * (size_t)s);
    double *of = (double *)malloc(sizeof(double) * (size_t)(s > 1 ? s - 1 : 1));
#pragma omp parallel for schedule(static)
    for (int64_t a = 0; a < s; ++a)
        for (int64_t b = 0; b < s; ++b) {
            double q = 0.0;
            for (int64_t t = 0; t < r; ++t) q = q + Lo[(r + a) * m + t] * Lo[(r + b) * m + t];
            E[a * s + b] = Ko[(r + a) * m + r + b] - q;
        }
    orc_tridiagonalize(E, s, dg, of);
    /* ||E_r||_2 < theta  <=>  every eigenvalue of E_r lies below theta */
    int below = (orc_sturm_count(dg, of, s, theta) == s);
    free(E); free(dg); free(of);
    return below;
}

int64_t orc_rank_estimate(const double *X, int64_t n, int d, int kernel, double l, double mu,
                          int64_t m, uint64_t seed, int64_t k_max, int64_t *r_out, int *branch_out)
{
    if (m > n) m = n;
    if (m < 1) m = 1;
    int64_t *sub = (int64_t *)malloc(sizeof(int64_t) * (size_t)m);
    orc_uniform_sample(n, m, seed, sub);
    double sc = pow((double)m / (double)n, 1.0 / (double)d);
    double *Xs = (double *)malloc(sizeof(double) * (size_t)(m * d));
    for (int64_t i = 0; i < m; ++i)
        for (int t = 0; t < d; ++t) Xs[i * d + t] = X[sub[i] * d + t] * sc;
    int64_t *o = (int64_t *)malloc(sizeof(int64_t) * (size_t)m);
    orc_fps(Xs, m, d, m, 0, o);
    double *Xo = (double *)malloc(sizeof(double) * (size_t)(m * d));
    for (int64_t i = 0; i < m; ++i)
        for (int t = 0; t < d; ++t) Xo[i * d + t] = Xs[o[i] * d + t];
    double *Ko = (double *)malloc(sizeof(double) * (size_t)(m * m));
    orc_kernel_matrix(Xo, m, Xo, m, d, kernel, l, Ko);
    /* ||K_m||_2 */
    double *T = (double *)malloc(sizeof(double) * (size_t)(m * m));
    double *dg = (double *)malloc(sizeof(double) * (size_t)m);
    double *of = (double *)malloc(sizeof(double) * (size_t)(m > 1 ? m - 1 : 1));
    memcpy(T, Ko, sizeof(double) * (size_t)(m * m));
    orc_tridiagonalize(T, m, dg, of);
    double lmax = orc_tridiag_max_eig(dg, of, m);
    double theta = 0.1 * lmax;
    /* Cholesky of K_m in FPS order with zero pivots dropped */
    double *Lo = (double *)calloc((size_t)(m * m), sizeof(double));
    double dmax = 0.0;
    for (int64_t i = 0; i < m; ++i) if (Ko[i * m + i] > dmax) dmax = Ko[i * m + i];
    double tiny = (double)m * 2.220446049250313e-16 * dmax;
    for (int64_t j = 0; j < m; ++j) {
        double s = Ko[j * m + j];
        for (int64_t p = 0; p < j; ++p) s = s - Lo[j * m + p] * Lo[j * m + p];
        if (!(s > tiny)) continue;                    /* column stays zero */
        double ljj = sqrt(s);
        Lo[j * m + j] = ljj;
#pragma omp parallel for schedule(static) if (m - j > 256)
        for (int64_t i = j + 1; i < m; ++i) {
            double t = Ko[i * m + j];
            for (int64_t p = 0; p < j; ++p) t = t - Lo[i * m + p] * Lo[j * m + p];
            Lo[i * m + j] = t / ljj;
        }
    }
    /* smallest r in [1, m] with ||E_r|| < theta (E_m is empty) */
    int64_t lo = 1, hi = m;
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (nys_error_below(Ko, Lo, m, mid, theta)) hi = mid; else lo = mid + 1;
    }
    int64_t r = lo;
    int64_t k;
    int branch;
    if (r * n >= 2000 * m) {
        k = (r * n + m - 1) / m;
        branch = 0;
    } else {
        double *Ku = (double *)malloc(sizeof(double) * (size_t)(m * m));
        double *Xu = (double *)malloc(sizeof(double) * (size_t)(m * d));
        for (int64_t i = 0; i < m; ++i)
            for (int t = 0; t < d; ++t) Xu[i * d + t] = X[sub[i] * d + t];
        orc_kernel_matrix(Xu, m, Xu, m, d, kernel, l, Ku);
        orc_tridiagonalize(Ku, m, dg, of);
        k = m - orc_sturm_count(dg, of, m, 0.1 * mu);
        branch = 1;
        free(Ku); free(Xu);
    }
    int64_t cap = k_max < n ? k_max : n;
    if (k > cap) k = cap;
    if (k < 1) k = 1;
    if (r_out) *r_out = r;
    if (branch_out) *branch_out = branch;
    free(sub); free(Xs); free(o); free(Xo); free(Ko); free(T); free(dg); free(of); free(Lo);
    return k;
}

/* ------------------------------------------------------------------------ */
/* Sampled outputs for large problems (same arithmetic as above, on a subset */
/* of rows).                                                                 */
/* ------------------------------------------------------------------------ */
/* y[r, c] = ((K + mu I) p)[rows[r], c], p n x nrhs column-major,
 * y nrows x nrhs column-major */
void orc_matvec_rows(const double *X, int64_t n, int d, int kernel, double l, double mu,
                     const double *p, int nrhs, const int64_t *rows, int64_t nrows, double *y)
{
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t q = 0; q < nrows; ++q) {
        int64_t i = rows[q];
        for (int c = 0; c < nrhs; ++c) {
            const double *pc = p + (int64_t)c * n;
            double s = 0.0;
            for (int64_t j = 0; j < n; ++j)
                s = s + orc_kernel_eval(X + i * d, X + j * d, d, kernel, l) * pc[j];
            y[(int64_t)c * nrows + q] = s + mu * pc[i];
        }
    }
}

/* FSAI rows of Alg. 1 on the Schur complement for selected Schur rows, with
 * the pattern given (nr x w) and K12 columns formed on the fly from the
 * permuted points Xp (landmarks first).  Same literal Schur block as
 * orc_afn_build.  G out: nrows x w.  Returns 0, 1 (a size or row index
 * out of range) or 3. */
int orc_fsai_rows(const double *Xp, int64_t n, int d, int kernel, double l, double mu, int64_t k,
                  int w, const double *L, const int32_t *pat, const int64_t *rows, int64_t nrows,
                  double *Gout)
{
    if (k < 0 || k > n || w < 1 || d < 1) return 1;
    for (int64_t q = 0; q < nrows; ++q)
        if (rows[q] < 0 || rows[q] >= n - k) return 1;
    const double *Xk = Xp, *Xr = Xp + k * d;
    int bad = 0;
#pragma omp parallel
    {
        double *Kc = (double *)malloc(sizeof(double) * (size_t)((k > 0 ? k : 1) * w));
        double *V = (double *)malloc(sizeof(double) * (size_t)((k > 0 ? k : 1) * w));
        double *tmp = (double *)malloc(sizeof(double) * (size_t)(k > 0 ? k : 1));
        double *A = (double *)malloc(sizeof(double) * (size_t)(w * w));
        double *g = (double *)malloc(sizeof(double) * (size_t)w);
#pragma omp for schedule(dynamic, 1)
        for (int64_t q = 0; q < nrows; ++q) {
            int64_t i = rows[q];
            const int32_t *s = pat + i * w;
            int m = 0;
            while (m < w && s[m] >= 0) ++m;
            for (int c = 0; c < m; ++c) {
                for (int64_t t = 0; t < k; ++t)
                    Kc[(int64_t)c * k + t] = orc_kernel_eval(Xk + t * d, Xr + (int64_t)s[c] * d, d, kernel, l);
                if (k > 0) {
                    orc_forward(L, k, Kc + (int64_t)c * k, tmp);
                    orc_backward(L, k, tmp, V + (int64_t)c * k);
                }
            }
            for (int a = 0; a < m; ++a)
                for (int b = 0; b < m; ++b) {
                    double v = orc_kernel_eval(Xr + (int64_t)s[a] * d, Xr + (int64_t)s[b] * d, d, kernel, l);
                    if (a == b) v = v + mu;
                    double qq = 0.0;
                    for (int64_t t = 0; t < k; ++t) qq = qq + Kc[(int64_t)a * k + t] * V[(int64_t)b * k + t];
                    A[a * m + b] = v - qq;
                }
            for (int p = 0; p < w; ++p) Gout[q * w + p] = 0.0;
            if (orc_fsai_row(A, m, g)) {
#pragma omp atomic write
                bad = 3;
            } else {
                for (int p = 0; p < m; ++p) Gout[q * w + p] = g[p];
            }
        }
        free(Kc); free(V); free(tmp); free(A); free(g);
    }
    return bad;
}
