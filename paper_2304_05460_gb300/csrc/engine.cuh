// engine.cuh -- host side of the grouped PCG: a Group owns the device
// description of its member systems (group.cuh), their solve workspaces and
// one captured CUDA graph that advances every member by `chunk` iterations of
// the mixed-precision PCG with reliable FP64 residual replacements.  Members
// can join and leave between graph launches (batched solves add all members
// up front; the serving loop admits and retires them continuously).
#pragma once

#include <cuda_runtime.h>

#include <vector>

#include "afn_internal.cuh"
#include "group.cuh"

namespace afn {

struct Member {
    Handle *h = nullptr;          // built factors (owned by the caller)
    int nrhs = 0, ncg = 0, js = 0;
    int64_t kch = 0;
    DevBuf ws;                    // vectors, apply temporaries, column states
    GSys desc{};
    int slot = -1;                // index in the device system array, -1 when not live
    bool fresh = false;           // columns still to be initialised
    bool done = false;
    void *tag = nullptr;          // owner's bookkeeping
};

class Group {
public:
    static constexpr int MAX_SYS = 1 << 16;
    static constexpr int NSTAGE = 5;   // profiled stages of an iteration

    // share: fraction of the GPU's CTA slots the persistent grids take
    Group(cudaStream_t s, int chunk, double tol, double delta, int maxit, double share = 1.0);
    ~Group();
    Group(const Group &) = delete;
    Group &operator=(const Group &) = delete;

    // Adds a built mixed-precision handle with nrhs right-hand sides b
    // (device, n x nrhs column-major, original point order).  The member
    // becomes live at the next step().
    afn_status add(Member *m, Handle *h, const double *b_dev, int nrhs);
    // One graph launch (chunk iterations of every live member); appends the
    // members whose columns have all stopped to `finished` (they stay in the
    // group, frozen, until remove()).
    afn_status step(std::vector<Member *> &finished);
    // x (device, n x nrhs, original order) and per-column iterations,
    // relative residuals and convergence flags (host arrays, may be NULL).
    afn_status collect(Member *m, double *x_dev, int32_t *iters, double *relres, int *conv);
    void remove(Member *m);
    int live() const;
    static size_t workspace_bytes(const Handle *h, int nrhs);

private:
    afn_status upload();
    afn_status capture();
    void tune();                  // persistent-grid sizes of the grouped kernels (autotuner)
    afn_status iteration(int it);
    void mark(int it, int stage);

    cudaStream_t strm_;
    int chunk_;
    double tol_, delta_;
    int maxit_;
    double share_;
    std::vector<Member *> mem_;
    bool dirty_ = true;
    // device buffers
    DevBuf gd_, sys_, tiles_, cols_, rep_, nact_, init_;
    int *nact_host_ = nullptr;
    cudaGraphExec_t exec_ = nullptr;
    long long kpg_ = 0;           // kernels per graph launch
    bool tuned_ = false;
    int cps_mv_ = 0, cps_ap_ = 0; // CTAs per SM of the grouped matvec and apply (0 = default)
    int launches_ = 0;
    GDev hgd_{};
    bool prof_ = false;
    std::vector<cudaEvent_t> ev_;
    double stage_ms_[NSTAGE] = {0, 0, 0, 0, 0};
    // host staging (kept until the next synchronisation)
    std::vector<GSys> hsys_;
    std::vector<GTile> htiles_;
    std::vector<int2> hcols_, hinit_;
};

// Builds systems on `threads` host threads (own non-blocking streams,
// largest first); hs[i] is system i's handle.  The streams must outlive the
// handles.
afn_status build_many(const afn_system *sys, int ns, const afn_options &o, int threads,
                      std::vector<Handle *> &hs, std::vector<cudaStream_t> &streams);
int build_threads(int ns);

}  // namespace afn
