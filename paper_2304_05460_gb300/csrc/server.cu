// server.cu -- the serving loop: solve requests of different n, d, kernel,
// l and mu arrive at any time; each is admitted when its device-memory
// footprint fits the budget, built by one of several host threads on its own
// stream (the builds overlap each other and the running solves on the GPU),
// then joins the running group of PCG solves (engine.cuh) at the next graph
// launch, and leaves it when all its columns have stopped.  Its solution is
// copied to host memory and every device buffer it held is released, which
// admits the next requests (continuous batching).
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "afn_internal.cuh"
#include "engine.cuh"

namespace afn {

using Clock = std::chrono::steady_clock;

static double ms_since(Clock::time_point a, Clock::time_point b)
{
    return std::chrono::duration<double, std::milli>(b - a).count();
}

// AFN_LOG_BUILD=1: host wall times of the serving steps on stderr (diagnostics)
static bool log_build()
{
    static const bool on = [] {
        const char *e = getenv("AFN_LOG_BUILD");
        return e && e[0] == '1';
    }();
    return on;
}

enum ReqState { RQ_QUEUED, RQ_BUILDING, RQ_READY, RQ_SOLVING, RQ_DONE };

struct Request {
    int64_t id = 0;
    afn_system sys{};
    std::vector<double> X, B;      // host copies of the points and right-hand sides
    int nrhs = 0;
    double tol = 1e-6;
    int64_t bytes = 0;             // reserved device-memory footprint
    ReqState state = RQ_QUEUED;
    afn_status status = AFN_OK;
    std::string error;
    Handle *h = nullptr;
    DevBuf bdev;                   // right-hand sides on the device (build stream)
    cudaStream_t bstream = nullptr;
    Member mem;
    std::vector<double> x;         // result (host)
    std::vector<int32_t> iters;
    std::vector<double> relres;
    int converged = 0;
    Clock::time_point t_submit, t_admit, t_built, t_join, t_done;
    double build_ms = 0;
};

// device bytes a request holds while admitted: its factors (mixed handle),
// the largest build temporaries and its grouped-solve workspace
static int64_t footprint(int64_t n, int d, int64_t kmax, int w, int nrhs, bool wide)
{
    const int64_t fw = wide ? 8 : 4;                      // factor element bytes
    const int64_t k = std::min<int64_t>(kmax, n), nr = n - k;
    const int64_t ww = std::max<int64_t>(1, std::min<int64_t>(w, std::max<int64_t>(nr, 1)));
    const int ds = d <= 4 ? 4 : (d <= 8 ? 8 : 16);
    int64_t b = 0;
    b += n * 8 + n * d * 8 + n * ds * 4;                  // perm, X64, X32
    b += k * k * 8 + 2 * k * k * fw;                     // L, L^{-1}, L^{-T}
    b += nr * k * fw;                                     // W^T
    b += nr * ww * (4 + 8 + 4) + (nr + 1 + 2 * nr * ww) * 4;   // pattern, G, G32, G^T lists
    b += k * k * 4 + n * d * 8 + nr * ww * 8 * 4;         // build temporaries (L32, input, FSAI)
    const int C = (nrhs + GC - 1) / GC * GC;
    const int64_t js = nr > 0 ? (nr + 2047) / 2048 : 0;
    b += n * C * (3 * 8 + 5 * 4) + 2 * k * C * 4 + 2 * nr * C * 4 + js * C * k * 4 + C * 128;
    b += (n + 64) * (ds + 2) * 8 + (n + 64) * C * 20;    // staged point and p tiles
    b += n * nrhs * 8;                                    // rhs upload
    return b + (4 << 20);                                 // allocator granularity, small arrays
}

struct Server {
    int dev = 0;
    afn_options opt{};
    int64_t budget = 0;
    int max_active = 0;
    int nbuild = 8;
    cudaStream_t stream = nullptr;

    std::mutex mu;
    std::condition_variable cv_sched, cv_build, cv_done, cv_single;
    bool stop = false;
    int64_t next_id = 1;
    std::deque<Request *> queue;           // submitted, not admitted
    std::deque<Request *> to_build;        // admitted, waiting for a build thread
    std::vector<Request *> ready;          // built, waiting to join the group
    std::deque<Request *> single;          // built DF requests, waiting for a solver thread
    std::map<int64_t, Request *> all;
    std::deque<int64_t> completed;         // done, not yet reported by poll
    int64_t reserved = 0, peak_reserved = 0;
    int active = 0;                        // admitted and not done
    int64_t n_submitted = 0, n_done = 0, graph_launches = 0;
    int peak_live = 0;

    std::thread sched;
    std::vector<std::thread> builders, singles;
    std::vector<cudaStream_t> bstreams, sstreams;
    int nsingle = 6;
    std::atomic<double> df_share{1.0};    // GPU share of a one-at-a-time solve's matvec

    void build_loop(int t);
    void single_loop(int t);
    void sched_loop();
    void finish(Request *r, Group *g);
};

void Server::build_loop(int t)
{
    cudaSetDevice(dev);
    cudaStream_t s = bstreams[t];
    for (;;) {
        Request *r = nullptr;
        {
            std::unique_lock<std::mutex> lk(mu);
            cv_build.wait(lk, [&] { return stop || !to_build.empty(); });
            if (stop) return;
            r = to_build.front();
            to_build.pop_front();
        }
        auto t0 = Clock::now();
        afn_options o = opt;
        o.stream = s;
        Handle *h = nullptr;
        afn_status st = create_handle(r->X.data(), r->sys.n, r->sys.d, r->sys.kernel, r->sys.l,
                                      r->sys.mu, r->sys.k_max, r->sys.fsai_nnz, o, s, &h);
        std::string err = st == AFN_OK ? "" : afn_last_error();
        const auto t1 = Clock::now();
        if (st == AFN_OK) {
            StreamGuard sg(s);
            const size_t bytes = sizeof(double) * r->B.size();
            st = r->bdev.alloc(bytes);
            if (st == AFN_OK) {
                cudaError_t e = cudaMemcpyAsync(r->bdev.p, r->B.data(), bytes, cudaMemcpyHostToDevice, s);
                if (e == cudaSuccess) e = cudaStreamSynchronize(s);
                if (e != cudaSuccess) st = cuda_fail(e, "request rhs upload");
            }
            if (st != AFN_OK) err = afn_last_error();
        }
        if (log_build()) {
            const auto t2 = Clock::now();
            fprintf(stderr, "[afn serve] request %lld n=%lld: create %.1f ms, rhs upload %.1f ms\n",
                    (long long)r->id, (long long)r->sys.n, ms_since(t0, t1), ms_since(t1, t2));
        }
        if (st == AFN_OK && h->precision != AFN_PREC_MIXED) {
            // a DF (or FP64) request -- AFN_PREC_AUTO's choice for a small mu --
            // goes to the one-at-a-time solver threads, so builds keep flowing
            {
                std::lock_guard<std::mutex> lk(mu);
                r->t_built = Clock::now();
                r->build_ms = ms_since(t0, r->t_built);
                r->h = h;
                r->bstream = s;
                r->state = RQ_READY;
                single.push_back(r);
            }
            cv_single.notify_one();
            continue;
        }
        {
            std::lock_guard<std::mutex> lk(mu);
            r->h = h;
            r->bstream = s;
            r->status = st;
            r->error = err;
            r->t_built = Clock::now();
            r->build_ms = ms_since(t0, r->t_built);
            r->state = RQ_READY;
            ready.push_back(r);
        }
        cv_sched.notify_one();
    }
}

// One-at-a-time solves of the DF (or FP64) requests, on low-priority streams
// of their own beside the running group and the builds.
void Server::single_loop(int t)
{
    cudaSetDevice(dev);
    cudaStream_t s = sstreams[t];
    for (;;) {
        Request *r = nullptr;
        {
            std::unique_lock<std::mutex> lk(mu);
            cv_single.wait(lk, [&] { return stop || !single.empty(); });
            if (stop) return;
            r = single.front();
            single.pop_front();
            r->t_join = Clock::now();
        }
        Handle *h = r->h;
        h->stream = s;
        StreamGuard sg(s);
        GridShareGuard gs(&df_share);   // the group keeps free SMs for its short kernels
        DevBuf xd;
        r->iters.assign(r->nrhs, 0);
        r->relres.assign(r->nrhs, 0.0);
        int outer = 0, conv = 0;
        afn_status st = xd.alloc(sizeof(double) * r->sys.n * r->nrhs);
        if (st == AFN_OK)
            st = solve_handle(h, r->bdev.as<double>(), r->nrhs, r->tol, xd.as<double>(),
                              r->iters.data(), r->relres.data(), &outer, &conv);
        if (st == AFN_OK || st == AFN_ERR_NO_CONVERGE) {
            r->x.resize((size_t)r->sys.n * r->nrhs);
            cudaError_t e = cudaMemcpyAsync(r->x.data(), xd.p, sizeof(double) * r->x.size(),
                                            cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) st = cuda_fail(e, "request result copy");
        }
        r->converged = conv;
        r->status = st;
        r->error = st == AFN_OK ? "" : (st == AFN_ERR_NO_CONVERGE ? "some columns missed tol"
                                                                 : afn_last_error());
        finish(r, nullptr);
    }
}

// Result to host, device memory released, reservation returned.
void Server::finish(Request *r, Group *g)
{
    if (r->state == RQ_SOLVING && g) {
        DevBuf xd;
        {
            StreamGuard sg(stream);
            afn_status st = xd.alloc(sizeof(double) * r->sys.n * r->nrhs);
            std::vector<int> conv(r->nrhs, 0);
            r->iters.assign(r->nrhs, 0);
            r->relres.assign(r->nrhs, 0.0);
            if (st == AFN_OK)
                st = g->collect(&r->mem, xd.as<double>(), r->iters.data(), r->relres.data(), conv.data());
            if (st == AFN_OK) {
                r->x.resize((size_t)r->sys.n * r->nrhs);
                cudaError_t e = cudaMemcpyAsync(r->x.data(), xd.p, sizeof(double) * r->x.size(),
                                                cudaMemcpyDeviceToHost, stream);
                if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
                if (e != cudaSuccess) st = cuda_fail(e, "request result copy");
            }
            r->converged = 0;
            for (int c : conv) r->converged += c;
            if (st == AFN_OK && r->converged != r->nrhs) st = AFN_ERR_NO_CONVERGE;
            if (st != AFN_OK && r->status == AFN_OK) {
                r->status = st;
                r->error = st == AFN_ERR_NO_CONVERGE ? "some columns missed tol" : afn_last_error();
            }
        }
        g->remove(&r->mem);
        r->mem.ws.release();
    }
    cudaStreamSynchronize(stream);
    r->bdev.release();
    delete r->h;
    r->h = nullptr;
    r->X.clear();
    r->X.shrink_to_fit();
    r->B.clear();
    r->B.shrink_to_fit();
    std::lock_guard<std::mutex> lk(mu);
    r->state = RQ_DONE;
    r->t_done = Clock::now();
    reserved -= r->bytes;
    --active;
    ++n_done;
    completed.push_back(r->id);
    cv_done.notify_all();
}

void Server::sched_loop()
{
    cudaSetDevice(dev);
    const int maxit = opt.max_iter > 0 ? opt.max_iter : 500;
    const double delta = opt.inner_tol > 0 ? opt.inner_tol : 0.01;
    const int chunk = opt.check_every > 0 ? opt.check_every : 4;
    // one group per tolerance value (the tolerance is a group constant)
    std::map<double, Group *> groups;
    auto group_for = [&](double tol) {
        auto it = groups.find(tol);
        if (it != groups.end()) return it->second;
        // the group leaves about a third of the SMs' CTA slots to the builds
        // and one-at-a-time solves running beside it
        Group *g = new Group(stream, chunk, tol, delta, maxit, 0.65);
        groups[tol] = g;
        return g;
    };
    std::vector<Member *> fin;
    std::vector<Request *> solving;        // scheduler-owned list of joined requests
    for (;;) {
        std::vector<Request *> joining;
        {
            std::unique_lock<std::mutex> lk(mu);
            if (stop) break;
            // admission by device-memory footprint, in arrival order; a
            // request larger than the whole budget runs when nothing else does
            while (!queue.empty()) {
                Request *r = queue.front();
                const bool fits = reserved + r->bytes <= budget || active == 0;
                if (!fits || (max_active > 0 && active >= max_active)) break;
                queue.pop_front();
                reserved += r->bytes;
                peak_reserved = std::max(peak_reserved, reserved);
                ++active;
                r->state = RQ_BUILDING;
                r->t_admit = Clock::now();
                to_build.push_back(r);
                cv_build.notify_one();
            }
            joining.swap(ready);
            if (solving.empty() && joining.empty()) {
                df_share = 1.0;
                cv_sched.wait_for(lk, std::chrono::milliseconds(20));
                continue;
            }
        }
        for (Request *r : joining) {
            if (r->status == AFN_OK) {
                Group *g = group_for(r->tol);
                afn_status st = g->add(&r->mem, r->h, r->bdev.as<double>(), r->nrhs);
                if (st == AFN_OK) {
                    r->mem.tag = r;
                    r->state = RQ_SOLVING;
                    r->t_join = Clock::now();
                    solving.push_back(r);
                    continue;
                }
                r->status = st;
                r->error = afn_last_error();
            }
            finish(r, nullptr);
        }
        int live = 0;
        for (auto &kv : groups) {
            Group *g = kv.second;
            if (g->live() == 0) continue;
            fin.clear();
            afn_status st = g->step(fin);
            ++graph_launches;
            live += g->live() + (int)fin.size();
            std::vector<Request *> ended;
            for (Member *m : fin) ended.push_back(static_cast<Request *>(m->tag));
            if (st != AFN_OK) {
                // a failed launch ends every request of this group with its error
                const std::string msg = afn_last_error();
                for (Request *r : solving)
                    if (r->tol == kv.first && std::find(ended.begin(), ended.end(), r) == ended.end()) {
                        r->status = st;
                        r->error = msg;
                        ended.push_back(r);
                    }
            }
            for (Request *r : ended) {
                finish(r, g);
                solving.erase(std::remove(solving.begin(), solving.end(), r), solving.end());
            }
        }
        peak_live = std::max(peak_live, live);
        // a one-at-a-time solve takes a fifth of the CTA slots while the group
        // has members (its short kernels then find free SMs), all otherwise
        df_share = live > 0 ? 0.2 : 1.0;
    }
    for (auto &kv : groups) delete kv.second;
}

}  // namespace afn

using namespace afn;

extern "C" {

void afn_server_default_config(afn_server_config *c)
{
    if (!c) return;
    memset(c, 0, sizeof(*c));
    afn_default_options(&c->opt);
    c->opt.precision = AFN_PREC_AUTO;
    c->build_threads = 8;
}

afn_status afn_server_create(const afn_server_config *cfg, afn_server **out)
{
    if (!out) { set_error("afn_server_create: out is NULL"); return AFN_ERR_ARG; }
    *out = nullptr;
    afn_server_config c;
    afn_server_default_config(&c);
    if (cfg) c = *cfg;
    if (c.opt.precond != AFN_PRECOND_AFN) {
        set_error("afn_server_create: served solves take the AFN preconditioner only (precond=%d)",
                  c.opt.precond);
        return AFN_ERR_ARG;
    }
    if (c.opt.precision < AFN_PREC_FP64 || c.opt.precision > AFN_PREC_AUTO) {
        set_error("afn_server_create: bad precision %d", c.opt.precision);
        return AFN_ERR_ARG;
    }
    if (c.memory_budget < 0 || c.max_active < 0 || c.build_threads < 0) {
        set_error("afn_server_create: negative limit");
        return AFN_ERR_ARG;
    }
    Server *s = new Server();
    cudaGetDevice(&s->dev);
    s->opt = c.opt;
    s->max_active = c.max_active;
    s->nbuild = c.build_threads > 0 ? c.build_threads : 8;
    size_t fr = 0, tot = 0;
    cudaMemGetInfo(&fr, &tot);
    s->budget = c.memory_budget > 0 ? c.memory_budget : (int64_t)(fr / 2);
    // builds get the highest stream priority (their many short kernels are
    // not held back by the long ones), the group the middle, DF solves the lowest
    int lo = 0, hi = 0;
    cudaDeviceGetStreamPriorityRange(&lo, &hi);
    if (cudaStreamCreateWithPriority(&s->stream, cudaStreamNonBlocking, (lo + hi) / 2) != cudaSuccess) {
        delete s;
        set_error("afn_server_create: stream creation failed");
        return AFN_ERR_CUDA;
    }
    s->bstreams.resize(s->nbuild);
    for (auto &b : s->bstreams) cudaStreamCreateWithPriority(&b, cudaStreamNonBlocking, hi);
    s->sstreams.resize(s->nsingle);
    for (auto &b : s->sstreams) cudaStreamCreateWithPriority(&b, cudaStreamNonBlocking, lo);
    for (int t = 0; t < s->nbuild; ++t) s->builders.emplace_back(&Server::build_loop, s, t);
    for (int t = 0; t < s->nsingle; ++t) s->singles.emplace_back(&Server::single_loop, s, t);
    s->sched = std::thread(&Server::sched_loop, s);
    *out = reinterpret_cast<afn_server *>(s);
    return AFN_OK;
}

afn_status afn_server_submit(afn_server *ss, const afn_system *sys, const double *rhs,
                             int32_t nrhs, double tol, int64_t *id)
{
    Server *s = reinterpret_cast<Server *>(ss);
    if (!s || !sys || !rhs || !id || nrhs < 1 || !(tol > 0) || !sys->points || sys->n < 1 ||
        sys->d < 1 || sys->d > 16) {
        set_error("afn_server_submit: invalid argument");
        return AFN_ERR_ARG;
    }
    Request *r = new Request();
    r->sys = *sys;
    r->nrhs = nrhs;
    r->tol = tol;
    const size_t nx = (size_t)sys->n * sys->d, nb = (size_t)sys->n * nrhs;
    r->X.resize(nx);
    r->B.resize(nb);
    cudaSetDevice(s->dev);
    auto fetch = [](void *dst, const void *src, size_t bytes) {
        if (!is_device_ptr(src)) {
            memcpy(dst, src, bytes);
            return true;
        }
        return cudaMemcpy(dst, src, bytes, cudaMemcpyDeviceToHost) == cudaSuccess;
    };
    if (!fetch(r->X.data(), sys->points, sizeof(double) * nx) ||
        !fetch(r->B.data(), rhs, sizeof(double) * nb)) {
        cudaGetLastError();
        delete r;
        set_error("afn_server_submit: cannot read points or rhs");
        return AFN_ERR_ARG;
    }
    for (double v : r->X)
        if (!std::isfinite(v)) { delete r; set_error("afn_server_submit: points contain NaN or Inf"); return AFN_ERR_ARG; }
    for (double v : r->B)
        if (!std::isfinite(v)) { delete r; set_error("afn_server_submit: rhs contains NaN or Inf"); return AFN_ERR_ARG; }
    r->sys.points = r->X.data();
    r->bytes = footprint(sys->n, sys->d, sys->k_max, sys->fsai_nnz, nrhs,
                         s->opt.precision != AFN_PREC_MIXED);
    r->t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        r->id = s->next_id++;
        s->all[r->id] = r;
        s->queue.push_back(r);
        ++s->n_submitted;
        *id = r->id;
    }
    s->cv_sched.notify_one();
    return AFN_OK;
}

afn_status afn_server_poll(afn_server *ss, int64_t *ids, int32_t max, int32_t *count,
                           int32_t wait_ms)
{
    Server *s = reinterpret_cast<Server *>(ss);
    if (!s || !count || (max > 0 && !ids)) {
        set_error("afn_server_poll: invalid argument");
        return AFN_ERR_ARG;
    }
    std::unique_lock<std::mutex> lk(s->mu);
    if (s->completed.empty() && wait_ms > 0)
        s->cv_done.wait_for(lk, std::chrono::milliseconds(wait_ms),
                            [&] { return !s->completed.empty(); });
    int c = 0;
    while (c < max && !s->completed.empty()) {
        ids[c++] = s->completed.front();
        s->completed.pop_front();
    }
    *count = c;
    return AFN_OK;
}

afn_status afn_server_result(afn_server *ss, int64_t id, double *x_out, int32_t *iters,
                             double *relres, afn_request_info *info)
{
    Server *s = reinterpret_cast<Server *>(ss);
    if (!s) { set_error("afn_server_result: invalid argument"); return AFN_ERR_ARG; }
    Request *r = nullptr;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        auto it = s->all.find(id);
        if (it == s->all.end()) {
            set_error("afn_server_result: unknown request %lld", (long long)id);
            return AFN_ERR_ARG;
        }
        r = it->second;
        if (r->state != RQ_DONE) {
            set_error("afn_server_result: request %lld has not finished", (long long)id);
            return AFN_ERR_BUSY;
        }
        s->all.erase(it);
    }
    afn_status st = r->status;
    if (x_out && !r->x.empty()) {
        const size_t bytes = sizeof(double) * r->x.size();
        if (!is_device_ptr(x_out)) {
            memcpy(x_out, r->x.data(), bytes);
        } else if (cudaMemcpy(x_out, r->x.data(), bytes, cudaMemcpyHostToDevice) != cudaSuccess) {
            cudaGetLastError();
            if (st == AFN_OK) st = AFN_ERR_CUDA;
        }
    }
    for (int c = 0; c < (int)r->iters.size(); ++c) {
        if (iters) iters[c] = r->iters[c];
        if (relres) relres[c] = r->relres[c];
    }
    if (info) {
        info->status = r->status;
        info->converged = r->converged;
        info->nrhs = r->nrhs;
        info->queue_ms = ms_since(r->t_submit, r->t_admit);
        info->build_ms = r->build_ms;
        const bool joined = r->t_join.time_since_epoch().count() != 0;
        info->wait_ms = joined ? ms_since(r->t_built, r->t_join) : 0.0;
        info->solve_ms = joined ? ms_since(r->t_join, r->t_done) : 0.0;
        info->latency_ms = ms_since(r->t_submit, r->t_done);
        info->device_bytes = r->bytes;
    }
    if (st != AFN_OK) set_error("request %lld: %s", (long long)id, r->error.c_str());
    delete r;
    return st;
}

afn_status afn_server_get_stats(afn_server *ss, afn_server_stats *out)
{
    Server *s = reinterpret_cast<Server *>(ss);
    if (!s || !out) { set_error("afn_server_get_stats: invalid argument"); return AFN_ERR_ARG; }
    std::lock_guard<std::mutex> lk(s->mu);
    out->submitted = s->n_submitted;
    out->completed = s->n_done;
    out->queued = (int64_t)s->queue.size();
    out->active = s->active;
    out->peak_live = s->peak_live;
    out->graph_launches = s->graph_launches;
    out->reserved_bytes = s->reserved;
    out->peak_reserved_bytes = s->peak_reserved;
    out->budget_bytes = s->budget;
    return AFN_OK;
}

void afn_server_destroy(afn_server *ss)
{
    Server *s = reinterpret_cast<Server *>(ss);
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_build.notify_all();
    s->cv_sched.notify_all();
    s->cv_single.notify_all();
    for (auto &t : s->builders) t.join();
    for (auto &t : s->singles) t.join();
    if (s->sched.joinable()) s->sched.join();
    cudaStreamSynchronize(s->stream);
    for (auto &kv : s->all) {
        Request *r = kv.second;
        r->mem.ws.release();
        r->bdev.release();
        delete r->h;
        delete r;
    }
    for (auto b : s->bstreams) {
        cudaStreamSynchronize(b);
        cudaStreamDestroy(b);
    }
    for (auto b : s->sstreams) {
        cudaStreamSynchronize(b);
        cudaStreamDestroy(b);
    }
    cudaStreamDestroy(s->stream);
    delete s;
}

}  // extern "C"
