// group.cuh -- device-side description of a group of independent systems
// (K_s + mu_s I) a_s = b_s that advance their PCG iterations together: every
// step of the iteration is one launch over the tiles of all member systems
// (batched solves and the serving loop).  The kernels read the group through
// one device pointer, so the host can change the membership between launches
// of a captured CUDA graph without re-capturing it.
#pragma once

#include <stdint.h>

namespace afn {

static constexpr int GC = 8;          // right-hand-side columns per column group

struct GCol {                         // state of one right-hand-side column
    double rho, alpha, beta, bnorm, tolabs, rmax2, relres;
    int active, iters, conv, flag, first, pad;
};

struct GSys {                         // one member system
    int n, d, ds, k, nr, w, ncg, nrhs, kernel, js;
    int64_t kch;                      // rows of W^T per split-K chunk (js chunks)
    float mu32;
    double mu, l;
    const double *X64;                // n x d permuted points
    const float *X32;                 // n x ds prescaled points
    const float2 *Xdf;                // n x ds prescaled double-float points
    const unsigned long long *Xdup;   // npad x (ds + 2) duplicated FP32 pairs (staged tiles)
    uint32_t *Psp;                    // [ncg][npad][40] tf32 (hi, lo) split of p32 (staged tiles)
    int npad;                         // n rounded up to the 64-point tile
    const float *Linv, *LinvT, *Wt, *G;
    const int32_t *pat, *gptr, *grow, *gslot;
    double *b, *x, *q;                // n x C column-major (C = GC * ncg)
    float *x32, *r32, *q32, *z32, *p32;
    float *zp, *u;                    // k x C
    float *t, *y;                     // [ncg][nr][GC] row-major
    float *part;                      // [js][C][k] split-K partials of W s2
    GCol *cs;                         // C column states (columns >= nrhs are padding)
};

struct GTile {                        // one unit of work of a grouped launch
    int sys, cg, r0, aux;             // system, column group, first row, chunk
};

struct GDev {                         // the group, as the kernels see it
    GSys *sys;
    GTile *mv;   int nmv;             // 128-row tiles of the FP32 matvec
    GTile *mv64; int nmv64;           // 64-row tiles of the FP64 residual matvec
    GTile *kb;   int nkb;             // 128-row blocks of k (L^{-1}, L^{-T}, finish)
    GTile *wb;   int nwb;             // 128-row blocks of nr (W^T z')
    GTile *wtb;  int nwtb;            // (128-row block of k, chunk): W s2 partials
    GTile *sp;   int nsp;             // 32-row blocks of nr (G and G^T products)
    int2 *col;   int ncol;            // (system, column) of every real column
    int *rep;                         // per system: FP64 residual replacement now
    int *nact;                        // per system: active columns (status output)
    int *err;                         // set when a staged copy did not complete in time
    int nsys;
    int maxit;
    double tol, delta;
};

}  // namespace afn
