// batch.cu -- many independent systems solved together (the batched solve and
// the engine of the serving loop).
//
// Every member system runs the same mixed-precision PCG as a single mixed
// handle (Alg. 5 with the apply of Alg. 3): FP32 matvec, apply and vectors,
// FP64 scalars per column, x accumulated in FP64, and the recursive residual
// replaced by the FP64 residual b - (K + mu I) x once it has fallen by delta
// since the last replacement (reliable updates); a column stops when that
// FP64 residual is below tol ||b|| or after max_iter iterations.  Each step
// of an iteration is ONE launch over the tiles (matvec, apply) or columns
// (dots, updates) of all member systems, and `chunk` iterations are one
// captured CUDA graph.  A system's arithmetic never depends on the other
// members, so its result is the same alone and in any mix.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <numeric>
#include <string>
#include <thread>
#include <vector>

#include "afn_device.cuh"
#include "afn_internal.cuh"
#include "engine.cuh"
#include "matvec_tc.cuh"

namespace afn {

void count_launches(long long n);     // capi.cu: the library's launch counter

// ------------------------------------------------------ column kernels --
static constexpr int CB = 256;        // threads per column block

// block-wide sum in a fixed order; every thread returns the total
__device__ __forceinline__ double block_total(double v, double *red)
{
    v = warp_sum(v);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double s = 0.0;
    for (int w = 0; w < CB / 32; ++w) s += red[w];
    __syncthreads();
    return s;
}

// rho' = r.z; first iteration: p = z; else beta = rho'/rho, p = z + beta p
__global__ void __launch_bounds__(CB) gbeta_kernel(const GDev *__restrict__ gd)
{
    __shared__ double red[CB / 32];
    const int nc = gd->ncol;
    for (int ci = blockIdx.x; ci < nc; ci += gridDim.x) {
        const int2 sc = gd->col[ci];
        const GSys &S = gd->sys[sc.x];
        GCol &cs = S.cs[sc.y];
        if (!cs.active) continue;
        const int first = cs.first;
        const double rho = cs.rho;
        const int64_t n = S.n, off = (int64_t)sc.y * n;
        const float *r = S.r32 + off, *z = S.z32 + off;
        float *p = S.p32 + off;
        // the tf32 (hi, lo) split of p, staged by the grouped matvec
        uint32_t *psp = S.Psp + (int64_t)(sc.y / GC) * S.npad * TcRow<1>::ROW + sc.y % GC;
        double acc = 0.0;
        for (int64_t i = threadIdx.x; i < n; i += CB) acc += (double)r[i] * (double)z[i];
        const double v = block_total(acc, red);
        const float be = first ? 0.f : (float)(v / rho);
        for (int64_t i = threadIdx.x; i < n; i += CB) {
            const float pv = first ? z[i] : z[i] + be * p[i];
            p[i] = pv;
            uint32_t hi, lo;
            tf32_split(pv, hi, lo);
            psp[i * TcRow<1>::ROW] = hi;
            psp[i * TcRow<1>::ROW + TcRow<1>::PS] = lo;
        }
        if (threadIdx.x == 0) {
            if (!first) cs.beta = v / rho;
            cs.rho = v;
            cs.first = 0;
        }
    }
}

// alpha = rho / p.q
__global__ void __launch_bounds__(CB) galpha_kernel(const GDev *__restrict__ gd)
{
    __shared__ double red[CB / 32];
    const int nc = gd->ncol;
    for (int ci = blockIdx.x; ci < nc; ci += gridDim.x) {
        const int2 sc = gd->col[ci];
        const GSys &S = gd->sys[sc.x];
        GCol &cs = S.cs[sc.y];
        if (!cs.active) continue;
        const int64_t n = S.n, off = (int64_t)sc.y * n;
        const float *p = S.p32 + off, *q = S.q32 + off;
        double acc = 0.0;
        for (int64_t i = threadIdx.x; i < n; i += CB) acc += (double)p[i] * (double)q[i];
        const double v = block_total(acc, red);
        if (threadIdx.x == 0) {
            cs.alpha = cs.rho / v;
            cs.iters += 1;
        }
    }
}

// x32 += alpha p, r32 -= alpha q, then the reliable-update test on r.r
__global__ void __launch_bounds__(CB) gupdate_kernel(const GDev *__restrict__ gd)
{
    __shared__ double red[CB / 32];
    const int nc = gd->ncol;
    const double delta = gd->delta;
    const int maxit = gd->maxit;
    for (int ci = blockIdx.x; ci < nc; ci += gridDim.x) {
        const int2 sc = gd->col[ci];
        const GSys &S = gd->sys[sc.x];
        GCol &cs = S.cs[sc.y];
        if (!cs.active) continue;
        const float al = (float)cs.alpha;
        const int64_t n = S.n, off = (int64_t)sc.y * n;
        const float *p = S.p32 + off, *q = S.q32 + off;
        float *x = S.x32 + off, *r = S.r32 + off;
        double acc = 0.0;
        for (int64_t i = threadIdx.x; i < n; i += CB) {
            const float xv = x[i] + al * p[i];
            const float rv = r[i] - al * q[i];
            x[i] = xv;
            r[i] = rv;
            acc += (double)rv * (double)rv;
        }
        const double v = block_total(acc, red);
        if (threadIdx.x == 0) {
            if (v > cs.rmax2) cs.rmax2 = v;
            if (v <= delta * delta * cs.rmax2 || cs.iters >= maxit) cs.flag = 1;
        }
    }
}

// per system: replace the residual of every active column now if one asked
__global__ void grep_kernel(const GDev *__restrict__ gd)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= gd->nsys) return;
    const GSys &S = gd->sys[s];
    int any = 0;
    for (int c = 0; c < S.nrhs; ++c) any |= S.cs[c].active && S.cs[c].flag;
    gd->rep[s] = any;
}

// x += x32, x32 = 0 on the active columns of the replaced systems
__global__ void __launch_bounds__(CB) gacc_kernel(const GDev *__restrict__ gd)
{
    const int nc = gd->ncol;
    for (int ci = blockIdx.x; ci < nc; ci += gridDim.x) {
        const int2 sc = gd->col[ci];
        if (!gd->rep[sc.x]) continue;
        const GSys &S = gd->sys[sc.x];
        if (!S.cs[sc.y].active) continue;
        const int64_t n = S.n, off = (int64_t)sc.y * n;
        double *x = S.x + off;
        float *dx = S.x32 + off;
        for (int64_t i = threadIdx.x; i < n; i += CB) {
            x[i] += (double)dx[i];
            dx[i] = 0.f;
        }
    }
}

// r = b - q (q = (K + mu I) x in FP64), r32 = fl32(r), and the FP64 test
__global__ void __launch_bounds__(CB) gresid_kernel(const GDev *__restrict__ gd)
{
    __shared__ double red[CB / 32];
    const int nc = gd->ncol;
    const double tol = gd->tol;
    const int maxit = gd->maxit;
    for (int ci = blockIdx.x; ci < nc; ci += gridDim.x) {
        const int2 sc = gd->col[ci];
        if (!gd->rep[sc.x]) continue;
        const GSys &S = gd->sys[sc.x];
        GCol &cs = S.cs[sc.y];
        if (!cs.active) continue;
        const int64_t n = S.n, off = (int64_t)sc.y * n;
        const double *b = S.b + off, *q = S.q + off;
        float *r32 = S.r32 + off;
        double acc = 0.0;
        for (int64_t i = threadIdx.x; i < n; i += CB) {
            const double r = b[i] - q[i];
            r32[i] = (float)r;
            acc += r * r;
        }
        const double v = block_total(acc, red);
        if (threadIdx.x == 0) {
            const double bn = cs.bnorm;
            const double rel = bn > 0.0 ? sqrt(v) / bn : 0.0;
            cs.relres = rel;
            cs.flag = 0;
            if (rel <= tol) {
                cs.active = 0;
                cs.conv = 1;
            } else if (cs.iters >= maxit) {
                cs.active = 0;
                cs.conv = 0;
            } else {
                cs.rmax2 = v;
            }
        }
    }
}

// active columns per system (the host polls this after every graph launch)
__global__ void gstatus_kernel(const GDev *__restrict__ gd)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= gd->nsys) return;
    const GSys &S = gd->sys[s];
    int a = 0;
    for (int c = 0; c < S.nrhs; ++c) a += S.cs[c].active;
    gd->nact[s] = a;
}

// start of a new member's columns: ||b||, r32 = fl32(b), column state
// (x, x32, p32 are zero: the workspace is cleared when the member is added)
__global__ void __launch_bounds__(CB) ginit_kernel(const GDev *__restrict__ gd,
                                                   const int2 *__restrict__ cols, int ncols,
                                                   double delta)
{
    __shared__ double red[CB / 32];
    for (int ci = blockIdx.x; ci < ncols; ci += gridDim.x) {
        const int2 sc = cols[ci];
        const GSys &S = gd->sys[sc.x];
        GCol &cs = S.cs[sc.y];
        const int64_t n = S.n, off = (int64_t)sc.y * n;
        const double *b = S.b + off;
        float *r32 = S.r32 + off;
        double acc = 0.0;
        for (int64_t i = threadIdx.x; i < n; i += CB) {
            r32[i] = (float)b[i];
            acc += b[i] * b[i];
        }
        const double v = block_total(acc, red);
        if (threadIdx.x == 0) {
            const double bn = sqrt(v);
            cs.rho = cs.alpha = cs.beta = 0.0;
            cs.bnorm = bn;
            cs.tolabs = delta;
            cs.rmax2 = v;
            cs.relres = bn > 0.0 ? 1.0 : 0.0;
            cs.active = bn > 0.0 ? 1 : 0;
            cs.conv = bn > 0.0 ? 0 : 1;
            cs.iters = 0;
            cs.flag = 0;
            cs.first = 1;
        }
    }
}

static int sms()
{
    int dev = 0, v = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    return std::max(v, 1);
}

// ------------------------------------------------------------- Group --
static size_t al256(size_t b) { return (b + 255) / 256 * 256; }

static constexpr int64_t KCH = 2048;   // rows of W^T per split-K chunk

struct WsLayout {
    size_t b, x, q, x32, r32, q32, z32, p32, zp, u, t, y, part, cs, xdup, psp, total;
};

static WsLayout layout(int64_t n, int64_t k, int64_t nr, int C, int js, int ds)
{
    WsLayout L{};
    size_t o = 0;
    auto put = [&](size_t bytes) { size_t at = o; o += al256(bytes); return at; };
    const size_t v64 = sizeof(double) * (size_t)n * C, v32 = sizeof(float) * (size_t)n * C;
    L.b = put(v64);
    L.x = put(v64);
    L.q = put(v64);
    L.x32 = put(v32);
    L.r32 = put(v32);
    L.q32 = put(v32);
    L.z32 = put(v32);
    L.p32 = put(v32);
    L.zp = put(sizeof(float) * (size_t)k * C);
    L.u = put(sizeof(float) * (size_t)k * C);
    L.t = put(sizeof(float) * (size_t)nr * C);
    L.y = put(sizeof(float) * (size_t)nr * C);
    L.part = put(sizeof(float) * (size_t)js * C * (size_t)k);
    L.cs = put(sizeof(GCol) * (size_t)C);
    const size_t np = (size_t)group_npad(n);
    L.xdup = put(sizeof(unsigned long long) * np * (size_t)(ds + 2));
    L.psp = put(sizeof(uint32_t) * (size_t)(C / GC) * np * TcRow<1>::ROW);
    L.total = o;
    return L;
}

size_t Group::workspace_bytes(const Handle *h, int nrhs)
{
    const int ncg = (nrhs + GC - 1) / GC;
    const int js = h->nr > 0 ? (int)((h->nr + KCH - 1) / KCH) : 0;
    return layout(h->n, h->k, h->nr, ncg * GC, js, stored_dim32(h->dp)).total;
}

// AFN_GROUP_PROFILE=1: stage times of the grouped iteration from CUDA events
// recorded inside the captured graph, printed to stderr when the group ends
static const char *STAGE_NAMES[Group::NSTAGE] = {"apply", "beta/p", "matvec32", "alpha/update",
                                                 "residual"};

Group::Group(cudaStream_t s, int chunk, double tol, double delta, int maxit, double share)
    : strm_(s), chunk_(std::max(1, chunk)), tol_(tol), delta_(delta), maxit_(maxit),
      share_(share > 0 && share <= 1 ? share : 1.0)
{
    const char *e = getenv("AFN_GROUP_PROFILE");
    prof_ = e && e[0] == '1';
}

Group::~Group()
{
    if (prof_ && launches_ > 0) {
        fprintf(stderr, "[afn group] %d graph launches of %d iterations:", launches_, chunk_);
        for (int k = 0; k < NSTAGE; ++k) fprintf(stderr, " %s %.1f ms", STAGE_NAMES[k], stage_ms_[k]);
        fprintf(stderr, "\n");
    }
    for (auto e : ev_) cudaEventDestroy(e);
    if (exec_) cudaGraphExecDestroy(exec_);
    if (nact_host_) cudaFreeHost(nact_host_);
}

afn_status Group::add(Member *m, Handle *h, const double *b_dev, int nrhs)
{
    if (!h || h->precision != AFN_PREC_MIXED || nrhs < 1) {
        set_error("grouped solve: needs a mixed-precision handle and nrhs >= 1");
        return AFN_ERR_ARG;
    }
    StreamGuard sg(strm_);
    m->h = h;
    m->nrhs = nrhs;
    m->ncg = (nrhs + GC - 1) / GC;
    const int C = m->ncg * GC;
    m->kch = KCH;
    m->js = h->nr > 0 ? (int)((h->nr + KCH - 1) / KCH) : 0;
    const WsLayout L = layout(h->n, h->k, h->nr, C, m->js, stored_dim32(h->dp));
    AFN_TRY(m->ws.alloc(L.total));
    AFN_CUDA(cudaMemsetAsync(m->ws.p, 0, L.total, strm_));
    char *base = static_cast<char *>(m->ws.p);
    GSys &g = m->desc;
    memset(&g, 0, sizeof(g));
    g.n = (int)h->n;
    g.d = h->d;
    g.ds = stored_dim32(h->dp);
    g.k = (int)h->k;
    g.nr = (int)h->nr;
    g.w = h->w;
    g.ncg = m->ncg;
    g.nrhs = nrhs;
    g.kernel = h->kernel;
    g.js = m->js;
    g.kch = m->kch;
    g.mu32 = (float)h->mu;
    g.mu = h->mu;
    g.l = h->l;
    g.X64 = h->X64.as<double>();
    g.X32 = h->X32.as<float>();
    g.Xdf = h->Xdf.as<float2>();
    g.Linv = h->Linv32.as<float>();
    g.LinvT = h->LinvT32.as<float>();
    g.Wt = h->Wt32.as<float>();
    g.G = h->G32.as<float>();
    g.pat = h->pat.as<int32_t>();
    g.gptr = h->gt_ptr.as<int32_t>();
    g.grow = h->gt_row.as<int32_t>();
    g.gslot = h->gt_slot.as<int32_t>();
    g.b = reinterpret_cast<double *>(base + L.b);
    g.x = reinterpret_cast<double *>(base + L.x);
    g.q = reinterpret_cast<double *>(base + L.q);
    g.x32 = reinterpret_cast<float *>(base + L.x32);
    g.r32 = reinterpret_cast<float *>(base + L.r32);
    g.q32 = reinterpret_cast<float *>(base + L.q32);
    g.z32 = reinterpret_cast<float *>(base + L.z32);
    g.p32 = reinterpret_cast<float *>(base + L.p32);
    g.zp = reinterpret_cast<float *>(base + L.zp);
    g.u = reinterpret_cast<float *>(base + L.u);
    g.t = reinterpret_cast<float *>(base + L.t);
    g.y = reinterpret_cast<float *>(base + L.y);
    g.part = reinterpret_cast<float *>(base + L.part);
    g.cs = reinterpret_cast<GCol *>(base + L.cs);
    g.npad = group_npad(h->n);
    g.Xdup = reinterpret_cast<const unsigned long long *>(base + L.xdup);
    g.Psp = reinterpret_cast<uint32_t *>(base + L.psp);
    dup_points(h->X32.as<float>(), h->n, g.ds, g.npad, base + L.xdup, strm_);
    gather_cols(b_dev, h->perm.as<int64_t>(), h->n, nrhs, g.b, strm_);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "grouped solve: gather rhs");
    m->fresh = true;
    m->done = false;
    m->slot = -1;
    mem_.push_back(m);
    dirty_ = true;
    return AFN_OK;
}

void Group::remove(Member *m)
{
    mem_.erase(std::remove(mem_.begin(), mem_.end(), m), mem_.end());
    m->slot = -1;
    dirty_ = true;
}

int Group::live() const
{
    int c = 0;
    for (auto *m : mem_) c += !m->done;
    return c;
}

template <class T>
static afn_status ensure(DevBuf &b, size_t count)
{
    size_t need = sizeof(T) * std::max<size_t>(count, 1);
    if (b.bytes >= need) return AFN_OK;
    return b.alloc(std::max(need, b.bytes * 2));
}

// Rebuilds the system array, the tile lists (largest systems first, so the
// persistent CTAs take the longest tiles early) and the column list of the
// live members, and copies them to the device.
afn_status Group::upload()
{
    StreamGuard sg(strm_);
    std::vector<Member *> lv;
    for (auto *m : mem_)
        if (!m->done) lv.push_back(m);
    std::stable_sort(lv.begin(), lv.end(),
                     [](const Member *a, const Member *b) { return a->desc.n > b->desc.n; });
    if ((int)lv.size() > MAX_SYS) {
        set_error("grouped solve: more than %d live systems", MAX_SYS);
        return AFN_ERR_ARG;
    }
    hsys_.clear();
    htiles_.clear();
    hcols_.clear();
    hinit_.clear();
    for (size_t i = 0; i < lv.size(); ++i) {
        lv[i]->slot = (int)i;
        hsys_.push_back(lv[i]->desc);
    }
    for (auto *m : mem_)
        if (m->done) m->slot = -1;
    const int R32 = group_mv32_rows(), R64 = group_mv64_rows(), RB = group_block_rows(),
              RS = group_sparse_rows();
    size_t seg[7];
    auto emit = [&](int which) {
        seg[which] = htiles_.size();
        for (size_t i = 0; i < lv.size(); ++i) {
            const GSys &g = lv[i]->desc;
            for (int cg = 0; cg < g.ncg; ++cg) {
                switch (which) {
                case 0: for (int r = 0; r < g.n; r += R32) htiles_.push_back({(int)i, cg, r, 0}); break;
                case 1: for (int r = 0; r < g.n; r += R64) htiles_.push_back({(int)i, cg, r, 0}); break;
                case 2: for (int r = 0; r < g.k; r += RB) htiles_.push_back({(int)i, cg, r, 0}); break;
                case 3: for (int r = 0; r < g.nr; r += RB) htiles_.push_back({(int)i, cg, r, 0}); break;
                case 4:
                    for (int q = 0; q < g.js; ++q)
                        for (int r = 0; r < g.k; r += RB) htiles_.push_back({(int)i, cg, r, q});
                    break;
                default: for (int r = 0; r < g.nr; r += RS) htiles_.push_back({(int)i, cg, r, 0}); break;
                }
            }
        }
    };
    for (int w = 0; w < 6; ++w) emit(w);
    seg[6] = htiles_.size();
    for (size_t i = 0; i < lv.size(); ++i) {
        for (int c = 0; c < lv[i]->nrhs; ++c) {
            hcols_.push_back(make_int2((int)i, c));
            if (lv[i]->fresh) hinit_.push_back(make_int2((int)i, c));
        }
        lv[i]->fresh = false;
    }
    AFN_TRY(ensure<GSys>(sys_, hsys_.size()));
    AFN_TRY(ensure<GTile>(tiles_, htiles_.size()));
    AFN_TRY(ensure<int2>(cols_, hcols_.size()));
    AFN_TRY(ensure<int2>(init_, hinit_.size()));
    if (!rep_.p) AFN_TRY(rep_.alloc(sizeof(int) * MAX_SYS));
    if (!nact_.p) {
        AFN_TRY(nact_.alloc(sizeof(int) * (MAX_SYS + 1)));   // + the staging status word
        AFN_CUDA(cudaMemsetAsync(nact_.p, 0, sizeof(int) * (MAX_SYS + 1), strm_));
    }
    if (!gd_.p) AFN_TRY(gd_.alloc(sizeof(GDev)));
    if (!hsys_.empty())
        AFN_CUDA(cudaMemcpyAsync(sys_.p, hsys_.data(), sizeof(GSys) * hsys_.size(), cudaMemcpyHostToDevice, strm_));
    if (!htiles_.empty())
        AFN_CUDA(cudaMemcpyAsync(tiles_.p, htiles_.data(), sizeof(GTile) * htiles_.size(), cudaMemcpyHostToDevice, strm_));
    if (!hcols_.empty())
        AFN_CUDA(cudaMemcpyAsync(cols_.p, hcols_.data(), sizeof(int2) * hcols_.size(), cudaMemcpyHostToDevice, strm_));
    if (!hinit_.empty())
        AFN_CUDA(cudaMemcpyAsync(init_.p, hinit_.data(), sizeof(int2) * hinit_.size(), cudaMemcpyHostToDevice, strm_));
    GTile *T = tiles_.as<GTile>();
    GDev h{};
    h.sys = sys_.as<GSys>();
    h.mv = T + seg[0];   h.nmv = (int)(seg[1] - seg[0]);
    h.mv64 = T + seg[1]; h.nmv64 = (int)(seg[2] - seg[1]);
    h.kb = T + seg[2];   h.nkb = (int)(seg[3] - seg[2]);
    h.wb = T + seg[3];   h.nwb = (int)(seg[4] - seg[3]);
    h.wtb = T + seg[4];  h.nwtb = (int)(seg[5] - seg[4]);
    h.sp = T + seg[5];   h.nsp = (int)(seg[6] - seg[5]);
    h.col = cols_.as<int2>();
    h.ncol = (int)hcols_.size();
    h.rep = rep_.as<int>();
    h.nact = nact_.as<int>();
    h.err = nact_.as<int>() + MAX_SYS;
    h.nsys = (int)hsys_.size();
    h.maxit = maxit_;
    h.tol = tol_;
    h.delta = delta_;
    hgd_ = h;
    AFN_CUDA(cudaMemcpyAsync(gd_.p, &hgd_, sizeof(GDev), cudaMemcpyHostToDevice, strm_));
    dirty_ = false;
    return AFN_OK;
}

void Group::mark(int it, int stage)
{
    if (!prof_) return;
    cudaEventRecord(ev_[(size_t)it * NSTAGE + stage], strm_);
}

afn_status Group::iteration(int it)
{
    const GDev *gd = gd_.as<GDev>();
    const int gc = persistent_grid(8, share_);
    mark(it, 0);
    AFN_TRY(group_apply(gd, strm_, share_, cps_ap_));              // z = M^{-1} r
    mark(it, 1);
    gbeta_kernel<<<gc, CB, 0, strm_>>>(gd);                // rho, beta, p
    mark(it, 2);
    AFN_TRY(group_matvec32(gd, strm_, share_, cps_mv_));           // q = (K + mu I) p
    mark(it, 3);
    galpha_kernel<<<gc, CB, 0, strm_>>>(gd);
    gupdate_kernel<<<gc, CB, 0, strm_>>>(gd);              // x, r, reliable-update test
    mark(it, 4);
    grep_kernel<<<MAX_SYS / 256, 256, 0, strm_>>>(gd);
    gacc_kernel<<<gc, CB, 0, strm_>>>(gd);                 // x += dx on replaced systems
    AFN_TRY(group_matvec64(gd, strm_, share_));                    // q = (K + mu I) x in FP64
    gresid_kernel<<<gc, CB, 0, strm_>>>(gd);               // r = b - q, FP64 test
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? AFN_OK : cuda_fail(e, "grouped iteration launch");
}

// The persistent grids' CTAs per SM, by the autotuner: the grouped matvec and
// apply are idempotent (their outputs are functions of p and r alone) and
// every tile is computed the same way by whichever CTA takes it, so the
// candidates are timed on the live group before the first iteration.
void Group::tune()
{
    tuned_ = true;
    const GDev *gd = gd_.as<GDev>();
    const std::string dev = tune_device_tag();
    static const int mvc[3] = {2, 3, 4}, apc[3] = {2, 4, 6};
    char key[96];
    snprintf(key, sizeof(key), "gmv32/tiles2^%d/%s", log2_bucket(hgd_.nmv), dev.c_str());
    cps_mv_ = mvc[tune_pick(key, 3, [&](int c) { group_matvec32(gd, strm_, share_, mvc[c]); }, strm_, 1)];
    snprintf(key, sizeof(key), "gapply/tiles2^%d/%s", log2_bucket(hgd_.nwb + hgd_.nsp), dev.c_str());
    cps_ap_ = apc[tune_pick(key, 3, [&](int c) { group_apply(gd, strm_, share_, apc[c]); }, strm_, 1)];
}

afn_status Group::capture()
{
    if (!nact_host_) AFN_CUDA(cudaMallocHost(&nact_host_, sizeof(int) * (MAX_SYS + 1)));
    const long long c0 = afn_launch_count();
    AFN_CUDA(cudaStreamBeginCapture(strm_, cudaStreamCaptureModeThreadLocal));
    afn_status st = AFN_OK;
    for (int it = 0; it < chunk_ && st == AFN_OK; ++it) st = iteration(it);
    if (st == AFN_OK) {
        gstatus_kernel<<<MAX_SYS / 256, 256, 0, strm_>>>(gd_.as<GDev>());
        cudaError_t e = cudaMemcpyAsync(nact_host_, nact_.p, sizeof(int) * (MAX_SYS + 1),
                                        cudaMemcpyDeviceToHost, strm_);
        if (e != cudaSuccess) st = cuda_fail(e, "grouped status copy");
    }
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(strm_, &g);
    if (st != AFN_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
    }
    if (e != cudaSuccess) return cuda_fail(e, "grouped graph capture");
    e = cudaGraphInstantiate(&exec_, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(e, "grouped graph instantiate");
    kpg_ = afn_launch_count() - c0;
    count_launches(-kpg_);      // captured, not launched
    return AFN_OK;
}

afn_status Group::step(std::vector<Member *> &finished)
{
    if (dirty_) AFN_TRY(upload());
    if (!hinit_.empty()) {
        ginit_kernel<<<sms() * 8, CB, 0, strm_>>>(gd_.as<GDev>(), init_.as<int2>(), (int)hinit_.size(),
                                               delta_);
        hinit_.clear();
    }
    if (hsys_.empty()) return AFN_OK;
    if (!tuned_) tune();
    if (prof_) {
        // profiling: the same launches issued eagerly between timing events
        if (!nact_host_) AFN_CUDA(cudaMallocHost(&nact_host_, sizeof(int) * (MAX_SYS + 1)));
        if (ev_.empty()) {
            ev_.resize((size_t)chunk_ * NSTAGE + 1);
            for (auto &e : ev_) cudaEventCreate(&e);
        }
        for (int it = 0; it < chunk_; ++it) AFN_TRY(iteration(it));
        cudaEventRecord(ev_.back(), strm_);
        gstatus_kernel<<<MAX_SYS / 256, 256, 0, strm_>>>(gd_.as<GDev>());
        AFN_CUDA(cudaMemcpyAsync(nact_host_, nact_.p, sizeof(int) * (MAX_SYS + 1),
                                 cudaMemcpyDeviceToHost, strm_));
    } else {
        if (!exec_) AFN_TRY(capture());
        AFN_CUDA(cudaGraphLaunch(exec_, strm_));
        count_launches(kpg_);
    }
    ++launches_;
    AFN_CUDA(cudaStreamSynchronize(strm_));
    if (prof_) {
        for (int it = 0; it < chunk_; ++it)
            for (int k = 0; k < NSTAGE; ++k) {
                float ms = 0;
                cudaEventElapsedTime(&ms, ev_[(size_t)it * NSTAGE + k], ev_[(size_t)it * NSTAGE + k + 1]);
                stage_ms_[k] += ms;
            }
    }
    if (nact_host_[MAX_SYS]) {
        set_error("grouped matvec: a staged tile copy did not complete in time");
        return AFN_ERR_TIMEOUT;
    }
    for (auto *m : mem_) {
        if (m->done || m->slot < 0) continue;
        if (nact_host_[m->slot] == 0) {
            m->done = true;
            finished.push_back(m);
            dirty_ = true;
        }
    }
    return AFN_OK;
}

afn_status Group::collect(Member *m, double *x_dev, int32_t *iters, double *relres, int *conv)
{
    const Handle *h = m->h;
    if (x_dev) scatter_cols(m->desc.x, h->perm.as<int64_t>(), h->n, m->nrhs, x_dev, strm_);
    std::vector<GCol> cs(m->nrhs);
    AFN_CUDA(cudaMemcpyAsync(cs.data(), m->desc.cs, sizeof(GCol) * m->nrhs, cudaMemcpyDeviceToHost, strm_));
    AFN_CUDA(cudaStreamSynchronize(strm_));
    for (int c = 0; c < m->nrhs; ++c) {
        if (iters) iters[c] = cs[c].iters;
        if (relres) relres[c] = cs[c].relres;
        if (conv) conv[c] = cs[c].conv;
    }
    return AFN_OK;
}

// ------------------------------------------------------- batched build --
struct Batch {
    int dev = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    afn_options opt{};
    std::vector<cudaStream_t> bstreams;    // build streams (the handles' buffers live on them)
    std::vector<Handle *> h;
    double build_ms = 0;
    ~Batch()
    {
        if (stream) cudaStreamSynchronize(stream);
        for (auto *x : h) delete x;
        for (auto s : bstreams) {
            cudaStreamSynchronize(s);
            cudaStreamDestroy(s);
        }
        if (own_stream && stream) cudaStreamDestroy(stream);
    }
};

// Builds systems [0, ns) on `threads` host threads, each with its own
// non-blocking stream, largest n first.  On failure every handle built so
// far is kept in hs (the caller frees them) and the first error is returned.
afn_status build_many(const afn_system *sys, int ns, const afn_options &o, int threads,
                      std::vector<Handle *> &hs, std::vector<cudaStream_t> &streams)
{
    int dev = 0;
    cudaGetDevice(&dev);
    hs.assign(ns, nullptr);
    std::vector<int> order(ns);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return sys[a].n > sys[b].n; });
    threads = std::max(1, std::min(threads, ns));
    streams.assign(threads, nullptr);
    std::atomic<int> next{0};
    std::atomic<bool> failed{false};
    std::mutex mu;
    afn_status first = AFN_OK;
    std::string msg;
    auto work = [&](int t) {
        cudaSetDevice(dev);
        if (cudaStreamCreateWithFlags(&streams[t], cudaStreamNonBlocking) != cudaSuccess) {
            std::lock_guard<std::mutex> lk(mu);
            if (first == AFN_OK) { first = AFN_ERR_CUDA; msg = "stream creation failed"; }
            failed = true;
            return;
        }
        for (;;) {
            if (failed) return;
            int i = next.fetch_add(1);
            if (i >= ns) return;
            const afn_system &y = sys[order[i]];
            Handle *h = nullptr;
            afn_status st = create_handle(y.points, y.n, y.d, y.kernel, y.l, y.mu, y.k_max,
                                          y.fsai_nnz, o, streams[t], &h);
            if (st != AFN_OK) {
                std::lock_guard<std::mutex> lk(mu);
                if (first == AFN_OK) {
                    first = st;
                    msg = "system " + std::to_string(order[i]) + ": " + afn_last_error();
                }
                failed = true;
                return;
            }
            hs[order[i]] = h;
        }
    };
    std::vector<std::thread> pool;
    for (int t = 1; t < threads; ++t) pool.emplace_back(work, t);
    work(0);
    for (auto &th : pool) th.join();
    if (first != AFN_OK) set_error("%s", msg.c_str());
    return first;
}

int build_threads(int ns)
{
    const char *e = getenv("AFN_BUILD_THREADS");
    int t = e ? atoi(e) : 16;
    return std::max(1, std::min(t, ns));
}

}  // namespace afn

using namespace afn;

extern "C" {

afn_status afn_build_batched(const afn_system *systems, int32_t nsys, const afn_options *opt,
                             afn_batch **out)
{
    if (!out || !systems || nsys < 1) {
        set_error("afn_build_batched: invalid argument");
        return AFN_ERR_ARG;
    }
    *out = nullptr;
    afn_options o;
    afn_default_options(&o);
    if (opt) o = *opt;
    if (o.precond != AFN_PRECOND_AFN) {
        set_error("afn_build_batched: grouped solves take the AFN preconditioner only (precond=%d)",
                  o.precond);
        return AFN_ERR_ARG;
    }
    Batch *b = new Batch();
    cudaGetDevice(&b->dev);
    b->opt = o;
    if (o.stream) {
        b->stream = static_cast<cudaStream_t>(o.stream);
    } else {
        if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete b;
            set_error("afn_build_batched: stream creation failed");
            return AFN_ERR_CUDA;
        }
        b->own_stream = true;
    }
    auto t0 = std::chrono::steady_clock::now();
    afn_status st = build_many(systems, nsys, o, build_threads(nsys), b->h, b->bstreams);
    if (st != AFN_OK) {
        delete b;
        return st;
    }
    for (auto s : b->bstreams) cudaStreamSynchronize(s);
    b->build_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    *out = reinterpret_cast<afn_batch *>(b);
    return AFN_OK;
}

afn_status afn_solve_batched(afn_batch *bb, const double *rhs, const int32_t *nrhs, double tol,
                             double *x_out, int32_t *iters, double *relres,
                             afn_batch_solve_info *info)
{
    Batch *b = reinterpret_cast<Batch *>(bb);
    if (!b || !rhs || !nrhs || !x_out || !(tol > 0) || !std::isfinite(tol)) {
        set_error("afn_solve_batched: invalid argument");
        return AFN_ERR_ARG;
    }
    const int ns = (int)b->h.size();
    std::vector<int64_t> off(ns + 1, 0), coff(ns + 1, 0);
    for (int s = 0; s < ns; ++s) {
        if (nrhs[s] < 1) {
            set_error("afn_solve_batched: nrhs[%d] < 1", s);
            return AFN_ERR_ARG;
        }
        off[s + 1] = off[s] + b->h[s]->n * nrhs[s];
        coff[s + 1] = coff[s] + nrhs[s];
    }
    cudaStream_t s = b->stream;
    StreamGuard sg(s);
    const int64_t tot = off[ns];
    DevBuf rin, xo, flag;
    const double *R = nullptr;
    AFN_TRY(to_device(rhs, tot, rin, &R, s));
    AFN_TRY(flag.alloc(sizeof(int)));
    AFN_TRY(check_finite(R, tot, flag.as<int>(), s, "rhs"));
    const bool xdev = is_device_ptr(x_out);
    double *X = x_out;
    if (!xdev) {
        AFN_TRY(xo.alloc(sizeof(double) * tot));
        X = xo.as<double>();
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, s);
    const int maxit = b->opt.max_iter > 0 ? b->opt.max_iter : 500;
    const double delta = b->opt.inner_tol > 0 ? b->opt.inner_tol : 0.01;
    const int chunk = b->opt.check_every > 0 ? b->opt.check_every : 4;
    afn_status st = AFN_OK;
    int launches = 0;
    std::vector<int> conv(coff[ns], 0);
    std::vector<int32_t> it(coff[ns], 0);
    std::vector<double> rel(coff[ns], 0.0);
    // systems whose handle is not mixed (DF or FP64, e.g. chosen by
    // AFN_PREC_AUTO for a small mu) are solved one at a time on the build
    // streams by host threads, overlapping the grouped solve of the others
    double group_ms = 0;
    std::atomic<double> df_share{0.5};    // 1 once the group has finished
    const auto w0 = std::chrono::steady_clock::now();
    std::atomic<long long> single_end_us{0};
    std::vector<int> single;
    for (int q = 0; q < ns; ++q)
        if (b->h[q]->precision != AFN_PREC_MIXED) single.push_back(q);
    // longest first (cost ~ n^2 x columns), so the last system to start is a short one
    std::stable_sort(single.begin(), single.end(), [&](int a, int c) {
        return (double)b->h[a]->n * (double)b->h[a]->n * nrhs[a] >
               (double)b->h[c]->n * (double)b->h[c]->n * nrhs[c];
    });
    std::vector<afn_status> sst(ns, AFN_OK);
    std::vector<int> sconv(ns, 0);
    std::atomic<int> snext{0};
    auto solo = [&](int t) {
        cudaSetDevice(b->dev);
        for (;;) {
            const int i = snext.fetch_add(1);
            if (i >= (int)single.size()) return;
            const int q = single[i];
            Handle *h = b->h[q];
            h->stream = b->bstreams[t % b->bstreams.size()];
            GridShareGuard gs(&df_share);   // the group keeps free SMs for its short kernels
            int outer = 0;
            sst[q] = solve_handle(h, R + off[q], nrhs[q], tol, X + off[q], it.data() + coff[q],
                                  rel.data() + coff[q], &outer, &sconv[q]);
            const long long us = std::chrono::duration_cast<std::chrono::microseconds>(
                                     std::chrono::steady_clock::now() - w0).count();
            long long prev = single_end_us.load();
            while (us > prev && !single_end_us.compare_exchange_weak(prev, us)) {
            }
        }
    };
    std::vector<std::thread> pool;
    const int nsolo = std::min<int>({(int)single.size(), (int)b->bstreams.size(), 8});
    for (int t = 0; t < nsolo; ++t) pool.emplace_back(solo, t);
    {
        std::vector<Member> mem(ns);
        Group g(s, chunk, tol, delta, maxit);
        for (int q = 0; q < ns && st == AFN_OK; ++q)
            if (b->h[q]->precision == AFN_PREC_MIXED) st = g.add(&mem[q], b->h[q], R + off[q], nrhs[q]);
        // every column stops by max_iter (a forced replacement), so the loop
        // ends; the bound below only guards against a logic error
        const int cap = (maxit + chunk) / chunk + 4;
        std::vector<Member *> fin;
        while (st == AFN_OK && g.live() > 0) {
            if (launches >= cap) {
                set_error("afn_solve_batched: columns still active after %d iterations", launches * chunk);
                st = AFN_ERR_NO_CONVERGE;
                break;
            }
            st = g.step(fin);
            ++launches;
        }
        group_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - w0).count();
        df_share = 1.0;
        for (int q = 0; q < ns && st == AFN_OK; ++q)
            if (b->h[q]->precision == AFN_PREC_MIXED)
                st = g.collect(&mem[q], X + off[q], it.data() + coff[q], rel.data() + coff[q],
                               conv.data() + coff[q]);
        for (auto &th : pool) th.join();
        for (int q : single) {
            for (int c = 0; c < nrhs[q]; ++c) conv[coff[q] + c] = rel[coff[q] + c] <= tol ? 1 : 0;
            if (st == AFN_OK && sst[q] != AFN_OK && sst[q] != AFN_ERR_NO_CONVERGE) st = sst[q];
        }
        if (st == AFN_OK && !xdev)
            st = cudaMemcpyAsync(x_out, X, sizeof(double) * tot, cudaMemcpyDeviceToHost, s) == cudaSuccess
                     ? AFN_OK : cuda_fail(cudaGetLastError(), "copy x_out");
        cudaStreamSynchronize(s);
    }
    cudaEventRecord(e1, s);
    cudaEventSynchronize(e1);
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != AFN_OK) return st;
    int nconv = 0, imax = 0;
    for (int64_t c = 0; c < coff[ns]; ++c) {
        nconv += conv[c];
        imax = std::max(imax, it[c]);
        if (iters) iters[c] = it[c];
        if (relres) relres[c] = rel[c];
    }
    if (info) {
        info->converged = nconv;
        info->columns = (int32_t)coff[ns];
        info->graph_launches = launches;
        info->iters_max = imax;
        info->solve_ms = ms;
        info->group_ms = group_ms;
        info->single_ms = single_end_us.load() / 1e3;
        info->single_systems = (int32_t)single.size();
    }
    if (nconv != coff[ns]) {
        set_error("afn_solve_batched: %d of %lld columns reached tol", nconv, (long long)coff[ns]);
        return AFN_ERR_NO_CONVERGE;
    }
    return AFN_OK;
}

afn_status afn_batch_build_info(const afn_batch *bb, int32_t system, afn_build_info *info)
{
    const Batch *b = reinterpret_cast<const Batch *>(bb);
    if (!b || !info || system < 0 || system >= (int)b->h.size()) {
        set_error("afn_batch_build_info: invalid argument");
        return AFN_ERR_ARG;
    }
    return afn_get_build_info(reinterpret_cast<const afn_handle *>(b->h[system]), info);
}

double afn_batch_build_ms(const afn_batch *bb)
{
    const Batch *b = reinterpret_cast<const Batch *>(bb);
    return b ? b->build_ms : 0.0;
}

void afn_batch_free(afn_batch *bb)
{
    delete reinterpret_cast<Batch *>(bb);
}

}  // extern "C"
