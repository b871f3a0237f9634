#!/usr/bin/env python3
"""AFN-PCG benchmark: solves/s at relative residual 1e-6 on one GB300.

Workload (default): the 8-D normal point set -- n = 50,000 points i.i.d.
N(0, I_8), Gaussian kernel, mu = 1e-2, landmark count estimated by Alg. 4 and
capped at 4000, FSAI with 64 nonzeros per row, 32 right-hand sides
b ~ N(0, 1), tol 1e-6.  One step = build + solve for each length-scale
l in {0.5, 1, 2, 4} (4 systems x 32 right-hand sides = 128 solves), mixed
precision (FP32 matvec / apply / FSAI Gram, FP64 Cholesky and triangular
inverse, FP64 dots and scalars, residual replacements by the FP64-accurate
double-float matvec).  The inputs (50,000 x 8 points, 50,000 x 32 RHS,
12.8 MB) are created once and stay resident in HBM; every step builds the
factors anew and the solve streams W^T (46,000 x 4,000 FP32 = 736 MB per
system) many times per step, far more than L2 (129 MB), so no L2 flush is
inserted between steps.

Output: one JSON line (rank 0).  ``--impl reference`` times the FP64 CPU
oracle (the reference arm) on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

LS = (0.5, 1.0, 2.0, 4.0)
N, D, MU, KMAX, W, NRHS, TOL, SEED = 50_000, 8, 1e-2, 4000, 64, 32, 1e-6, 1002
MAXIT = 3000   # per PCG solve; tol 1e-6 on these 8-D systems needs more than 500
SERVE_MAXIT = 1000   # per request in the serving stream (a request past it reports unconverged)
METRIC = "AFN-PCG solves/s at rel. residual 1e-6 (mixed precision, 8-D normal, n=50k, 32 RHS)"
PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")
N_SM, FP32_LANES, MUFU_PER_SM, SM_MAX_MHZ = 152, 128, 16, 2070.0
AUTO_RHO = [0.0]   # AFN_PREC_AUTO's MIXED/DF threshold for the batched and served systems (0 = 0.3)
LANE_PEAK_TOPS = N_SM * FP32_LANES * SM_MAX_MHZ * 1e6 / 1e12    # FP32 lane operations / s
# DRAM bytes read + written per launch of matvec32u_kernel<8, 4, Gaussian> at n = 50,000,
# 32 columns, from one ncu capture of that launch; to be re-taken when the kernel changes
MATVEC32_TRAFFIC_BYTES = 16048128 + 0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=N)
    ap.add_argument("--nrhs", type=int, default=NRHS)
    ap.add_argument("--e2e-steps", type=int, default=1)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--only", default="",
                    help="'batched', 'serving', 'clusters' or 'paper3d': run that workload alone")
    ap.add_argument("--paper-kernel", default="both", choices=["both", "gaussian", "matern"])
    ap.add_argument("--paper-kmax", type=int, default=20000)
    ap.add_argument("--paper-k", default="table", choices=["table", "estimate"])
    ap.add_argument("--paper-n", type=int, default=160_000)
    ap.add_argument("--paper-precision", default="auto", choices=["auto", "mixed", "df", "fp64"])
    ap.add_argument("--alg5-steps", type=int, default=1,
                    help="steps of the workload under the paper's Alg. 5 strategy (0 = skip)")
    ap.add_argument("--sequential", action="store_true",
                    help="build and solve the systems of a step one after another (default: "
                         "concurrently, one stream and host thread per system)")
    ap.add_argument("--ls", default="0.5,1,2,4",
                    help="length-scales of one step (a subset profiles a single system)")
    ap.add_argument("--batched", type=int, default=512,
                    help="systems of the batched workload (0 = skip)")
    ap.add_argument("--fp64-sample", type=int, default=24,
                    help="batched systems solved one at a time in plain FP64 for comparison")
    ap.add_argument("--serving", type=int, default=24,
                    help="requests of the serving stream (0 = skip)")
    ap.add_argument("--serving-rate", type=float, default=-0.8,
                    help="Poisson arrival rate, requests/s (0 = all requests at t = 0; "
                         "negative: that multiple of the measured FP64 one-at-a-time rate)")
    ap.add_argument("--auto-rho", type=float, default=0.0,
                    help="MIXED/DF threshold of AFN_PREC_AUTO for the batched and served "
                         "systems (0 = the library's 0.3)")
    ap.add_argument("--clusters", type=int, default=1,
                    help="1 = run the n = 200k clustered 64-RHS workload (0 = skip)")
    ap.add_argument("--one-rhs", type=int, default=1,
                    help="1 = run the n = 50k workload with one right-hand side (0 = skip)")
    return ap.parse_args()


def workload(n, nrhs):
    from paper_2304_05460_gb300 import inputs
    return inputs.normal_8d(l=1.0, nrhs=nrhs, n=n, seed=SEED)


def config(n, nrhs):
    return {"workload": "normal_8d: n=%d d=8 N(0,I), Gaussian l in {0.5,1,2,4}, mu=1e-2, "
                        "k=Alg.4 estimate capped at 4000, FSAI w=64, %d RHS N(0,1), tol 1e-6"
                        % (n, nrhs),
            "n": n, "d": D, "nrhs": nrhs, "lengthscales": list(LS), "mu": MU, "k_max": KMAX,
            "fsai_nnz": W, "tol": TOL, "precision": "mixed",
            "l2": "inputs and streamed factors far larger than L2 (129 MB); no flush"}


# ------------------------------------------------------------------ clocks --
class Clocks:
    def __init__(self, idx):
        self.idx = idx
        self.proc = None
        self.rows = []

    def start(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                                         text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        sm = [float(r[1]) for r in self.rows if len(r) >= 9 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if len(r) >= 9 and r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            if len(r) >= 9:
                for nm, v in zip(names, r[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(sm)}


# --------------------------------------------------------- oracle baseline --
# FP64 PCG iterations of the four systems of a step (tol 1e-6, 32 columns, max over the
# columns), as the FP64-accurate path measures them on the GPU; they only scale the oracle's
# sampled matvec time to whole solves (the oracle's own PCG would take hours at n = 50k)
FP64_ITERS = {0.5: 8, 1.0: 227, 2.0: 801, 4.0: 362}


# sizes of the oracle's bounded sample: "step" for each step of the reference arm (about 2 s
# on 16 host cores), "baseline" for the in-bench CPU baseline (about 10 s): FPS steps timed,
# landmarks of the timed Cholesky, FSAI rows with their literal Schur blocks, pattern rows of
# the timed KNN, matvec rows
SAMPLE_SIZES = {"step": dict(fps=400, kc=1200, fsai=8, knn=2000, mv=16),
                "baseline": dict(fps=2000, kc=2000, fsai=128, knn=4000, mv=1536)}


def oracle_sample(n, nrhs, size="step", iters_hint=None):
    """Time the FP64 oracle on a bounded sample of the workload (the l = 1
    system's build pieces and sampled matvec rows, sized by SAMPLE_SIZES[size])
    and scale to one step of the workload: one build per length-scale plus each
    system's PCG iterations.  Returns (solves_per_s, detail, cores, per-piece
    seconds)."""
    import oracle
    from paper_2304_05460_gb300 import inputs
    z = SAMPLE_SIZES[size]
    s = workload(n, nrhs)
    X = s.X
    l = 1.0
    cores = oracle.get_threads()
    t = {}
    t0 = time.perf_counter()
    k, r, br = oracle.rank_estimate(X, 0, l, MU, m=min(n, 1000), seed=SEED, k_max=KMAX)
    t["rank"] = time.perf_counter() - t0
    # FPS: the first steps of the k, scaled (each step is one O(n d) pass)
    ks = min(k, z["fps"])
    t0 = time.perf_counter()
    oracle.fps(X, ks, 0)
    t["fps"] = (time.perf_counter() - t0) * k / ks
    # Cholesky of K11 + mu I on the first kc landmarks, scaled by (k/kc)^3
    kc = min(k, z["kc"])
    idx = np.arange(kc)
    A = oracle.kernel_matrix(X[idx], X[idx], 0, l) + MU * np.eye(kc)
    t0 = time.perf_counter()
    Lc = oracle.cholesky(A)
    t["chol"] = (time.perf_counter() - t0) * (k / kc) ** 3
    # FSAI rows with their literal Schur blocks (full patterns), scaled to nr rows
    nr = n - k
    Xp = np.concatenate([X[:k], X[k:]])
    Lk = None
    if kc == k:
        Lk = Lc
    else:
        Ak = oracle.kernel_matrix(X[:k], X[:k], 0, l) + MU * np.eye(k)
        Lk = np.linalg.cholesky(Ak)      # factor only feeds the timed row solves below
    kr = min(nr, z["knn"])
    pat, _ = oracle.knn_pattern(Xp[k:k + kr], W)
    rows = np.arange(max(kr - 2 - z["fsai"], 0), kr - 2)
    t0 = time.perf_counter()
    oracle.fsai_rows(Xp, 0, l, MU, k, W, Lk,
                     np.concatenate([pat, np.full((nr - kr, W), -1, np.int32)]), rows)
    t["fsai"] = (time.perf_counter() - t0) * nr / len(rows)
    # KNN: rows 0..kr cost ~ sum i; scale to nr rows (quadratic)
    t0 = time.perf_counter()
    oracle.knn_pattern(Xp[k:k + kr], W)
    t["knn"] = (time.perf_counter() - t0) * (nr / float(kr)) ** 2
    # one PCG iteration ~ one matvec with nrhs columns: sampled rows scaled to n
    rowsm = np.arange(min(n, z["mv"]))
    P = inputs.rhs(n, nrhs, 5)
    t0 = time.perf_counter()
    oracle.matvec_rows(X, 0, l, MU, P, rowsm)
    t_mv = (time.perf_counter() - t0) * n / len(rowsm)
    # one build per system (sampled at l = 1) and each system's FP64 iteration count
    its = [FP64_ITERS.get(float(l), iters_hint or 227) for l in LS]
    build = sum(t.values())
    t["pcg"] = t_mv * sum(its)
    total = build * len(LS) + t["pcg"]
    detail = ("FP64 oracle, l=1 system: rank estimate in full; FPS %d of %d steps; Cholesky "
              "of %d of %d landmarks (x(k/kc)^3); %d FSAI rows of %d; KNN rows 0..%d "
              "(x(nr/%d)^2); %d matvec rows x %d RHS (x n); scaled to one step (the build "
              "once per system, PCG iterations %s for l = %s as the FP64-accurate GPU path "
              "counts them) = %.1f s" % (ks, k, kc, k, len(rows), nr, kr, kr, len(rowsm), nrhs,
                                        its, list(LS), total))
    return len(LS) * nrhs / total, detail, cores, t


# ------------------------------------------------------ replicas (N > 1) --
def job_time_ms(local_ms, dist, device):
    """The job's time: the maximum of the ranks' timed regions (every rank
    runs an independent replica of the workload, no data-path collective)."""
    if not dist:
        return local_ms
    import torch
    t = torch.tensor([float(local_ms)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(solves_per_rank, world, job_ms):
    """Whole-job solves/s: the solves of all ranks over the job's time."""
    return solves_per_rank * world / (job_ms / 1e3)


def deal(costs, world):
    """Independent systems dealt to ranks (replicas, no communication): the
    most expensive first, each to the rank with the least work so far (ties
    to the lower rank).  Returns one ascending index list per rank."""
    load = [0.0] * world
    share = [[] for _ in range(world)]
    for i in sorted(range(len(costs)), key=lambda j: (-costs[j], j)):
        r = min(range(world), key=lambda q: (load[q], q))
        share[r].append(i)
        load[r] += costs[i]
    return [sorted(x) for x in share]


def job_sum(value, dist, device):
    """Sum of a per-rank count over the ranks."""
    if not dist:
        return value
    import torch
    t = torch.tensor([float(value)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def job_gather(values, dist):
    """Every rank's list of values, concatenated in rank order."""
    if not dist:
        return list(values)
    parts = [None] * dist.get_world_size()
    dist.all_gather_object(parts, list(values))
    return [v for p in parts for v in p]


# ---------------------------------------------------------------- batched --
def run_batched(afn, count, fp64_sample, stream, rank=0, world=1, dist=None):
    """The batched workload: `count` systems (n log-uniform in [256, 8192],
    d in 2..16, N(0,I) points, Gaussian, l = median distance x log-uniform
    [0.1, 10], mu log-uniform [1e-4, 1e-1], k = min(n/4, 1000), w = 32, 8 RHS
    each), built and solved together (mixed precision, grouped kernels under
    CUDA graphs), against the plain FP64 GPU path run one system at a time on
    a seeded sample of the systems.  With several ranks the systems are dealt
    to them (``deal``, cost n^2) and each rank solves its share; the job's
    time is the slowest rank's."""
    import torch
    from paper_2304_05460_gb300 import inputs
    systems = inputs.batched_512(count=count)
    if world > 1:
        systems = [systems[i] for i in deal([float(x.n) ** 2 for x in systems], world)[rank]]
    args_ = [dict(points=torch.tensor(s.X, device="cuda"), kernel=s.kernel, l=s.l, mu=s.mu,
                  k_max=s.k, fsai_nnz=s.w) for s in systems]
    rhs = [torch.tensor(np.ascontiguousarray(s.B), device="cuda") for s in systems]
    cols = sum(s.nrhs for s in systems)
    opt = dict(seed=1004, max_iter=MAXIT, check_every=4, precision=afn.PREC_AUTO,
               auto_rho=AUTO_RHO[0])

    def once():
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        b = afn.afn_build_batched(args_, **opt)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        xs, info = afn.afn_solve_batched(b, rhs, TOL)
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        afn.afn_batch_free(b)
        return t1 - t0, t2 - t1, info

    once()                                   # warm-up (graph capture, pool growth)
    if dist:
        dist.barrier()
    bt, st, info = once()
    if dist:
        bt, st = job_time_ms(bt, dist, "cuda"), job_time_ms(st, dist, "cuda")
    # kernel-pair evaluations of the FP32 matvec: per system and column group,
    # n^2 pairs for every iteration in which one of its columns was active
    pairs = 0.0
    for s, its in zip(systems, info["iters"]):
        for g in range(0, len(its), 8):
            pairs += float(s.n) ** 2 * int(its[g:g + 8].max())
    conv = info["converged"]
    if dist:
        cols = int(job_sum(cols, dist, "cuda"))
        conv = int(job_sum(conv, dist, "cuda"))
        pairs = job_sum(pairs, dist, "cuda")
    out = {"workload": "batched_512: %d systems, n log-uniform [256, 8192], d in 2..16, N(0,I), "
                       "Gaussian, l = median dist x logU[0.1, 10], mu logU[1e-4, 1e-1], "
                       "k = min(n/4, 1000), w = 32, 8 RHS, tol 1e-6" % count,
           "systems": count, "ranks": world, "columns": cols, "converged_columns": conv,
           "build_ms": bt * 1e3, "solve_ms": st * 1e3,
           "solves_per_s": cols / (bt + st), "solve_only_solves_per_s": cols / st,
           "iters_max": info["iters_max"], "graph_launches": info["graph_launches"],
           "group_ms": info["group_ms"], "df_systems": info["single_systems"],
           "df_ms": info["single_ms"], "matvec_pairs_per_s": pairs / st}
    if fp64_sample > 0 and world == 1:
        g = np.random.Generator(np.random.PCG64(7))
        pick = sorted(g.choice(count, size=min(fp64_sample, count), replace=False).tolist())
        o64 = afn.options(precision=afn.PREC_FP64, seed=1004, max_iter=MAXIT, stream=stream)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        c64 = 0
        for i in pick:
            h = afn.afn_build(args_[i]["points"], systems[i].kernel, systems[i].l, systems[i].mu,
                              systems[i].k, systems[i].w, o64)
            x, inf = afn.afn_solve(h, rhs[i], TOL)
            c64 += int(inf["converged"])
            afn.afn_free(h)
        torch.cuda.synchronize()
        t64 = time.perf_counter() - t0
        n2 = sum(float(systems[i].n) ** 2 for i in pick)
        n2_all = sum(float(s.n) ** 2 for s in systems)
        # scale the sample's time by the workload's sum of n^2 (the matvec cost)
        t_all = t64 * n2_all / n2
        out["fp64_one_at_a_time"] = {
            "solves_per_s": cols / t_all, "sample_systems": len(pick),
            "sample_converged_columns": c64, "sample_s": t64,
            "scaling": "sample time x sum(n^2) of all systems / sum(n^2) of the sample"}
        out["speedup_vs_fp64"] = out["solves_per_s"] / out["fp64_one_at_a_time"]["solves_per_s"]
    return out


# ---------------------------------------------------------------- serving --
def serving_fp64_baseline(afn, count, fp64_sample):
    """The plain FP64 GPU path, one request at a time, on a seeded sample of the
    serving stream's requests with n <= 20,000 (larger ones take minutes in
    FP64), scaled to the whole stream by sum(n^2).  The FP64 matvec's cost is
    n^2 per iteration but the iteration counts differ between requests, so the
    scaled figure is an estimate; the sample and the scaling are reported."""
    import torch
    from paper_2304_05460_gb300 import inputs
    # the sample is drawn from the first 64 requests of the stream whatever `count` is, so the
    # estimate does not move with the stream's length
    pool = inputs.serving_stream(count=max(count, 64), rate=1.0)
    reqs = pool[:count]
    small = [i for i, r in enumerate(pool[:64]) if r["n"] <= 20_000]
    g = np.random.Generator(np.random.PCG64(11))
    pick = sorted(g.choice(small, size=min(fp64_sample, len(small)), replace=False).tolist())
    o64 = afn.options(precision=afn.PREC_FP64, seed=1005, max_iter=SERVE_MAXIT)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    for i in pick:
        sy = inputs.serving_system(pool[i])
        h = afn.afn_build(sy.X, sy.kernel, sy.l, sy.mu, sy.k, sy.w, o64)
        afn.afn_solve(h, sy.B, TOL)
        afn.afn_free(h)
    torch.cuda.synchronize()
    t64 = time.perf_counter() - t1
    n2 = sum(float(pool[i]["n"]) ** 2 for i in pick)
    n2_all = sum(float(r["n"]) ** 2 for r in reqs)
    t_all = t64 * n2_all / n2
    cols = sum(r["nrhs"] for r in reqs)
    return {"solves_per_s": cols / t_all, "requests_per_s": count / t_all,
            "sample_requests": len(pick), "sample_n": [int(pool[i]["n"]) for i in pick],
            "sample_s": t64, "s_per_n2": t64 / n2,
            "scaling": "sample (requests with n <= 20000) time x sum(n^2) / sum(n^2) of the "
                       "sample; an estimate: iteration counts are not proportional to n^2"}


def fifo_latencies_ms(arrivals_s, service_s):
    """Latencies (ms) of requests served one at a time in arrival order: each
    starts when it has arrived and the previous one has finished."""
    free, out = 0.0, []
    for t, sv in zip(arrivals_s, service_s):
        free = max(free, t) + sv
        out.append((free - t) * 1e3)
    return np.array(out)


def run_serving(afn, count, rate, fp64_sample, rank=0, world=1, dist=None, fp64=None):
    """The serving workload: `count` requests of the Poisson stream (n
    log-uniform in [1e3, 1e5], d in {3, 8, 16}, N(0,I) points, Gaussian or
    Matern-3/2 50/50, l and mu drawn as in the batched workload, k =
    min(n/4, 1000), w = 32, 1..16 RHS, tol 1e-6) replayed against the serving
    loop; latency is submit -> result.  rate > 0: Poisson arrivals at that
    rate (requests/s); rate == 0: every request at once (saturation); rate < 0:
    Poisson at -rate x the plain FP64 one-at-a-time throughput (measured first,
    ``serving_fp64_baseline``).  With several ranks the requests are dealt to
    them (``deal``, cost n^2), each rank serves its share at the share's own
    arrival times, and the job's makespan is the slowest rank's."""
    import threading
    import torch
    from paper_2304_05460_gb300 import inputs
    if fp64 is None and fp64_sample > 0 and world == 1:
        fp64 = serving_fp64_baseline(afn, count, fp64_sample)
    factor = None
    if rate < 0:
        if not fp64:
            raise RuntimeError("a rate relative to FP64 needs the FP64 baseline")
        factor = -rate
        rate = factor * fp64["requests_per_s"]
    reqs = inputs.serving_stream(count=count, rate=rate if rate > 0 else 1.0)
    if world > 1:
        reqs = [reqs[i] for i in deal([float(r["n"]) ** 2 for r in reqs], world)[rank]]
    systems = [inputs.serving_system(r) for r in reqs]
    args_ = [dict(points=s.X, kernel=s.kernel, l=s.l, mu=s.mu, k_max=s.k, fsai_nnz=s.w)
             for s in systems]
    cols = sum(s.nrhs for s in systems)
    srv = afn.Server(seed=1005, max_iter=SERVE_MAXIT, build_threads=8, auto_rho=AUTO_RHO[0])
    # warm-up request (graph capture, pool growth), not counted
    wid = srv.submit(args_[0], systems[0].B, TOL)
    while not srv.poll(wait_ms=100):
        pass
    srv.result(wid)
    ids = {}
    if dist:
        dist.barrier()
    t0 = time.perf_counter()

    def feeder():
        for i, r in enumerate(reqs):
            if rate > 0:
                dt = r["t"] - (time.perf_counter() - t0)
                if dt > 0:
                    time.sleep(dt)
            ids[srv.submit(args_[i], systems[i].B, TOL)] = i

    th = threading.Thread(target=feeder)
    th.start()
    lat, conv, done, qms = [], 0, 0, []
    while done < len(reqs):
        for rid in srv.poll(wait_ms=50):
            x, info = srv.result(rid)
            lat.append(info["latency_ms"])
            qms.append(info["queue_ms"])
            conv += int(info["converged"])
            done += 1
    span = time.perf_counter() - t0
    th.join()
    st = srv.stats()
    srv.close()
    if dist:
        span = job_time_ms(span * 1e3, dist, "cuda") / 1e3
        cols = int(job_sum(cols, dist, "cuda"))
        conv = int(job_sum(conv, dist, "cuda"))
        lat = job_gather(lat, dist)
    lat = np.sort(np.array(lat))
    arrivals = ("Poisson %.3g/s (%.2f x the FP64 one-at-a-time rate)" % (rate, factor)
                if factor else "Poisson %.3g/s" % rate if rate > 0 else "all at t = 0 (saturation)")
    out = {"workload": "serving_stream: %d requests, n log-uniform [1e3, 1e5], d in {3,8,16}, "
                       "N(0,I), Gaussian/Matern-3/2 50/50, l = median dist x logU[0.1, 10], "
                       "mu logU[1e-4, 1e-1], k = min(n/4, 1000), w = 32, 1-16 RHS, tol 1e-6, "
                       "at most %d iterations; arrivals: %s" % (count, SERVE_MAXIT, arrivals),
           "requests": count, "ranks": world, "rate_per_s": rate, "columns": cols,
           "converged_columns": conv, "makespan_s": span,
           "requests_per_s": count / span, "solves_per_s": cols / span,
           "latency_p50_ms": float(np.percentile(lat, 50)),
           "latency_p99_ms": float(np.percentile(lat, 99)),
           "latency_max_ms": float(lat[-1]),
           "queue_p50_ms": float(np.percentile(qms, 50)) if qms else None,
           "peak_live": st["peak_live"], "graph_launches": st["graph_launches"],
           "peak_reserved_gb": st["peak_reserved_bytes"] / 2**30}
    if fp64:
        out["fp64_one_at_a_time"] = fp64
        if rate <= 0:
            # saturation: every request at once, so the throughput ratio means something
            out["speedup_vs_fp64"] = out["solves_per_s"] / fp64["solves_per_s"]
        else:
            out["throughput_note"] = ("arrival-limited: the stream offers %.3g requests/s, so "
                                      "requests_per_s follows the arrivals; compare latencies"
                                      % rate)
        if rate > 0 and world == 1:
            # the same arrivals served one at a time by the FP64 path (FIFO), with each
            # request's service time estimated as s_per_n2 x n^2 from the timed sample
            fl = np.sort(fifo_latencies_ms([r["t"] for r in reqs],
                                           [fp64["s_per_n2"] * float(r["n"]) ** 2 for r in reqs]))
            out["fp64_fifo_estimate"] = {
                "latency_p50_ms": float(np.percentile(fl, 50)),
                "latency_p99_ms": float(np.percentile(fl, 99)),
                "basis": "FIFO queue over the same arrival times, service time = s_per_n2 x n^2 "
                         "(an estimate from the FP64 sample)"}
            out["latency_ratio_vs_fp64_fifo"] = {
                "p50": out["fp64_fifo_estimate"]["latency_p50_ms"] / out["latency_p50_ms"],
                "p99": out["fp64_fifo_estimate"]["latency_p99_ms"] / out["latency_p99_ms"]}
    return out


# ---------------------------------------------------- n = 200k clustered --
def hbm_peak():
    """(GB/s, basis) of the HBM roofline: the measured copy bandwidth."""
    try:
        with open(PEAKS) as f:
            return float(json.load(f)["hbm_gbs"]), "MEASURED_PEAKS.json hbm_gbs (measured copy)"
    except Exception:
        return 6800.0, "fallback 6.8 TB/s"


def run_clusters(afn, stream):
    """The clustered 3-D workload: n = 200,000 points (80 % in 3 Gaussian
    clusters, centres U[0,1]^3, sigma = 0.1, 20 % uniform), Matern-3/2 l = 0.05,
    mu = 1e-3, k = 2000 FPS landmarks, FSAI w = 50, 64 right-hand sides N(0,1),
    mixed precision with the BF16 tensor-core W products and FP64 residual
    replacements to tol 1e-6.  One build + solve timed with CUDA events after a
    warm-up on the first 20,000 points.  Rooflines: the FP32 matvec (FP32
    lane operations) and the apply (HBM bytes of its operators per apply)."""
    import torch
    from paper_2304_05460_gb300 import inputs
    s = inputs.clusters_3d(nrhs=64)
    Xd = torch.tensor(s.X, device="cuda")
    Bd = torch.tensor(np.ascontiguousarray(s.B), device="cuda")
    o = afn.options(precision=afn.PREC_MIXED, seed=1003, max_iter=MAXIT, stream=stream, profile=1)
    h = afn.afn_build(Xd[:20000].contiguous(), s.kernel, s.l, s.mu, 200, s.w, o)
    afn.afn_solve(h, Bd[:20000].contiguous(), TOL)
    afn.afn_free(h)
    torch.cuda.synchronize()
    e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    e[0].record(stream)
    h = afn.afn_build(Xd, s.kernel, s.l, s.mu, s.k, s.w, o)
    e[1].record(stream)
    x, info = afn.afn_solve(h, Bd, TOL)
    e[2].record(stream)
    torch.cuda.synchronize()
    bms, sms_ = e[0].elapsed_time(e[1]), e[1].elapsed_time(e[2])
    st = {nm: afn.afn_get_kernel_stats(h, nm) for nm in
          ("matvec32", "matvec64", "apply32", "blas1", "fps", "knn", "chol", "trsm", "fsai")}
    bi = h.info
    k, nr, w, n = int(bi.k), int(bi.nr), int(bi.w), int(bi.n)
    afn.afn_free(h)
    if info["converged"] != 64:
        raise RuntimeError("clusters_3d: %d/64 columns reached tol" % info["converged"])
    gbs, basis = hbm_peak()
    ap_cnt, ap_ms = st["apply32"]
    # algorithmic bytes of one 64-column apply: the BF16 W image read by each of the two
    # products, G (FP32 value + int32 index) by each sparse product, the triangular L^-1 and
    # L^-T (FP32), r read and s written once
    ap_bytes = 2 * 2.0 * k * nr + 2 * 8.0 * nr * w + 2 * 4.0 * k * (k + 1) / 2 + 2 * 4.0 * n * 64
    ap_avg = ap_ms / max(ap_cnt, 1)
    mv_cnt, mv_ms = st["matvec32"]
    mv_avg = mv_ms / max(mv_cnt, 1)          # one 64-column launch per matvec (tcgen05, N = 64)
    ops_pair = 2 * 4 + 4 + 64                # d-hat = 4: 2 d-hat + Matern's sqrt/scale + 64 columns
    mv_ops = float(n) * n * ops_pair
    return {"workload": "clusters_3d: n=200000 d=3 (3 clusters sigma=0.1 + 20%% uniform), "
                        "Matern-3/2 l=0.05, mu=1e-3, k=2000 FPS, w=50, 64 RHS N(0,1), tol 1e-6, "
                        "mixed precision, BF16 tensor-core W products",
            "value": 64.0 / ((bms + sms_) / 1e3), "unit": "solves/s",
            "solve_only_solves_per_s": 64.0 / (sms_ / 1e3), "build_ms": bms, "solve_ms": sms_,
            "iters_max": int(info["iters"].max()), "iters_mean": float(info["iters"].mean()),
            "residual_replacements": int(info["outer_steps"]),
            "relres_max": float(info["relres"].max()),
            "kernels": {a: {"launches": b[0], "ms": round(b[1], 3)} for a, b in st.items()},
            "roofline_apply": {"bound": "hbm", "achieved": ap_bytes / (ap_avg / 1e3) / 1e9,
                               "peak": gbs, "unit": "GB/s",
                               "frac": ap_bytes / (ap_avg / 1e3) / 1e9 / gbs,
                               "bytes_per_apply": ap_bytes, "avg_apply_ms": ap_avg,
                               "applies": ap_cnt, "peak_basis": basis},
            "roofline_matvec": {"bound": "alu", "achieved": mv_ops / (mv_avg / 1e3) / 1e12,
                                "peak": LANE_PEAK_TOPS, "unit": "Tops/s",
                                "frac": mv_ops / (mv_avg / 1e3) / 1e12 / LANE_PEAK_TOPS,
                                "ops_per_pair": ops_pair, "avg_matvec_ms": mv_avg,
                                "note": "the count takes one lane operation per column and pair "
                                        "for the contraction, which runs on the tensor cores, so "
                                        "the fraction can exceed 1; eval_bound is the FP32-pipe "
                                        "work that remains",
                                "eval_bound": {
                                    "pairs_per_s": float(n) * n / (mv_avg / 1e3),
                                    "peak_pairs_per_s": LANE_PEAK_TOPS * 1e12 / 12,
                                    "frac": float(n) * n / (mv_avg / 1e3) / (LANE_PEAK_TOPS * 1e12 / 12),
                                    "basis": "2 d-hat + 4 = 12 lane operations per Matern kernel "
                                             "value (d-hat = 4: differences, squares, sqrt, "
                                             "scale, exp, 1 + t)"}},
            "fp64_gpu": None,
            "fp64_note": "the plain FP64 GPU solve of this workload takes minutes (FP64 matvec "
                         "at n = 200k, 64 columns); measured once outside the default run"}


# ------------------------------------------------- the paper's 3-D cube --
# AFN iteration counts the paper prints for these columns (Table 1a, 1b); its runs
# use an H^2 matvec, other random points and FP64 arithmetic: context, not a target
PAPER_AFN_ITERS_GAUSSIAN = (3, 35, 37, 38, 40, 42, 46, 50, 57, 62, 1)
PAPER_AFN_ITERS_MATERN = (3, 6, 6, 6, 7, 7, 7, 7, 7, 6, 9)
# the rank k the paper's Alg. 4 estimated for each column (Table 1, row k)
PAPER_K_GAUSSIAN = (565, 9600, 9600, 9600, 9600, 12800, 12800, 12800, 16000, 19200, 160000)
PAPER_K_MATERN = (160000, 19200, 16000, 14080, 12800, 9600, 9600, 6400, 6400, 6400, 178)


def run_paper3d(afn, stream, which="both", k_max=20000, precision=None, kmode="table", n=160_000):
    """The paper's synthetic 3-D setting (Sec. 5, Table 1): n = 160,000 points
    U[0, n^(1/3)]^3, mu = 1e-4, one U[-0.5, 0.5] right-hand side, tol 1e-4,
    FSAI with w = 100, every Gaussian l^2 and Matern-3/2 1/l column of Table 1.
    kmode "table": the rank k the paper's Table 1 lists for the column (capped at
    k_max), with Alg. 5's rule on it (the Nystrom preconditioner below 2000, AFN
    above); kmode "estimate": this library's Alg. 4 estimate and Alg. 5.  Either
    way the Alg. 4 estimate is reported beside the paper's k.  Reports k, the
    branch, iterations, build and solve times per column beside the paper's
    AFN iterations."""
    import torch
    from paper_2304_05460_gb300 import inputs
    s = inputs.paper_cube_3d(n=n)
    Xd = torch.tensor(s.X, device="cuda")
    Bd = torch.tensor(np.ascontiguousarray(s.B), device="cuda")
    prec = afn.PREC_AUTO if precision is None else precision
    kscale = n / 160_000.0        # Table 1's k scaled to the same k / n on a smaller cube
    rows = []
    cases = []
    if which in ("both", "gaussian"):
        cases += [(afn.GAUSSIAN, "l2", v, float(np.sqrt(v)), p, kp) for v, p, kp in
                  zip(inputs.PAPER_GAUSSIAN_L2, PAPER_AFN_ITERS_GAUSSIAN, PAPER_K_GAUSSIAN)]
    if which in ("both", "matern"):
        cases += [(afn.MATERN32, "inv_l", v, 1.0 / v, p, kp) for v, p, kp in
                  zip(inputs.PAPER_MATERN_INV_L, PAPER_AFN_ITERS_MATERN, PAPER_K_MATERN)]
    for ker, lab, v, l, paper_it, paper_k in cases:
        k_est, r_est, br = afn.afn_rank_estimate(Xd, ker, l, s.mu, m=1000, seed=1006, k_max=k_max)
        if kmode == "table":
            k_use = min(max(1, int(round(paper_k * kscale))), k_max, n)
            pc = afn.PRECOND_NYSTROM if paper_k < 2000 else afn.PRECOND_AFN
            o = afn.options(precision=prec, precond=pc, seed=1006, max_iter=500, stream=stream)
        else:
            k_use = k_max
            o = afn.options(precision=prec, precond=afn.PRECOND_AUTO, rank_mode=afn.RANK_ESTIMATE,
                            rank_subsample=1000, seed=1006, max_iter=500, stream=stream)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        h = afn.afn_build(Xd, ker, l, s.mu, k_use, s.w, o)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        x, info = afn.afn_solve(h, Bd, 1e-4)
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        bi = h.info
        rows.append({"kernel": "gaussian" if ker == afn.GAUSSIAN else "matern32", lab: v,
                     "k": int(bi.k), "paper_k": paper_k, "alg4_k": int(k_est), "alg4_r": int(r_est),
                     "precision": {0: "fp64", 1: "mixed", 2: "df"}.get(int(bi.precision), "?"),
                     "rho32": float(bi.rho32),
                     "precond": "nystrom" if bi.precond == afn.PRECOND_NYSTROM else "afn",
                     "iters": int(info["iters"][0]), "converged": int(info["converged"]),
                     "relres": float(info["relres"][0]), "build_s": t1 - t0, "solve_s": t2 - t1,
                     "paper_afn_iters": paper_it})
        afn.afn_free(h)
        print(json.dumps(rows[-1]), file=sys.stderr, flush=True)
    return {"workload": "paper_cube_3d: n=%d U[0, n^(1/3)]^3, mu=1e-4, 1 RHS U[-0.5,0.5], "
                        "tol 1e-4, w=100, k %s (capped at %d)"
                        % (n, "from Table 1 scaled by n / 160000" if kmode == "table"
                           else "by Alg. 4 + Alg. 5", k_max),
            "precision": {afn.PREC_MIXED: "mixed", afn.PREC_AUTO: "auto (mixed or DF per system)",
                          afn.PREC_DF: "fp64-accurate (DF)", afn.PREC_FP64: "fp64"}[prec],
            "rows": rows,
            "note": "paper_afn_iters and paper_k: Table 1 of the paper (H^2 matvec, other points, "
                    "FP64); context only"}


# ------------------------------------------------------------ one column --
def run_one_rhs(afn, s, Xd, Bd, stream, opts):
    """The n = 50k, d = 8 workload with one right-hand side per system: the four
    length-scales built and solved concurrently (as the headline), one warm-up
    step and one timed step; the 1-column matvec runs on the CUDA cores
    (MUFU / FP32 bound) and its roofline is reported."""
    import torch
    st_ = [torch.cuda.Stream() for _ in LS]
    stats, iters = {}, []
    lock = threading.Lock()
    b1 = Bd[:, :1].contiguous()

    def one(l, st, prof):
        with torch.cuda.stream(st):
            h = afn.afn_build(Xd, afn.GAUSSIAN, l, MU, KMAX, W, opts(prof, st))
            x, info = afn.afn_solve(h, b1, TOL)
            st.synchronize()
        with lock:
            if info["converged"] != 1:
                raise RuntimeError("1 RHS, l=%g did not converge" % l)
            iters.append(int(info["iters"].max()))
            if prof:
                for nm in ("matvec32", "apply32"):
                    c, ms = afn.afn_get_kernel_stats(h, nm)
                    a = stats.setdefault(nm, [0, 0.0])
                    a[0] += c
                    a[1] += ms
        afn.afn_free(h)

    def step(prof):
        errs = []

        def run(l, st):
            try:
                one(l, st, prof)
            except BaseException as e:
                errs.append(e)
        ts = [threading.Thread(target=run, args=(l, st)) for l, st in zip(LS, st_)]
        for t in ts:
            t.start()
        for t in ts:
            t.join()
        if errs:
            raise errs[0]

    step(0)
    iters.clear()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    step(1)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    mv_cnt, mv_ms = stats.get("matvec32", [0, 0.0])
    avg = mv_ms / max(mv_cnt, 1)
    ops_pair = 2 * D + 1 + 1
    n = s.X.shape[0]
    ach = float(n) * n * ops_pair / (avg / 1e3) / 1e12
    mufu_peak = N_SM * MUFU_PER_SM * SM_MAX_MHZ * 1e6          # pairs/s at one EX2 a pair
    return {"workload": "normal_8d with 1 RHS per system (l in {0.5,1,2,4}, concurrent)",
            "value": len(LS) / (ms / 1e3), "unit": "solves/s", "ms_per_step": ms,
            "pcg_iters_max": iters,
            "roofline": {"bound": "alu", "achieved": ach, "peak": LANE_PEAK_TOPS, "unit": "Tops/s",
                         "frac": ach / LANE_PEAK_TOPS, "ops_per_pair": ops_pair,
                         "kernel": "matvec32r2_kernel<D=8,Gaussian> (CUDA cores, two rows per thread)",
                         "avg_launch_ms": avg, "launches": mv_cnt,
                         "mufu_bound_pairs_per_s": mufu_peak,
                         "pairs_per_s": float(n) * n / (avg / 1e3),
                         "note": "FP32 lane operations 2d+1+1 per pair; the EX2 (MUFU, "
                                 "16 per SM per cycle) bound is above the FP32 one at d = 8"}}


# ------------------------------------------------------------------- main --
def run_reference(args):
    """The reference arm: the FP64 oracle as it stands on the host cores.  Each
    step (warm-up steps included) is one bounded sample of the workload (the
    l = 1 system's build pieces and sampled matvec rows, SAMPLE_SIZES["step"]:
    about 2 s on 16 host cores); `ms_per_step` is the measured time of a timed step, `value` the
    sample's throughput scaled to the workload's solves (median over the timed
    steps).  Under torchrun only rank 0 runs."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    vals, secs = [], []
    detail, cores = "", 0
    for st in range(max(args.warmup, 0) + max(args.steps, 1)):
        t0 = time.perf_counter()
        v, detail, cores, _ = oracle_sample(args.n, args.nrhs)
        dt = time.perf_counter() - t0
        if st >= max(args.warmup, 0):
            vals.append(v)
            secs.append(dt)
    v = float(np.median(vals))
    step_ms = float(np.mean(secs)) * 1e3
    sample = ("each step one bounded sample of %.1f s (measured, ms_per_step); value = that "
              "sample scaled to the workload: %s" % (step_ms / 1e3, detail))
    line = {"metric": METRIC, "value": v, "unit": "solves/s", "n_gpus": args.gpus,
            "steps": len(secs), "warmup": args.warmup, "ms_per_step": step_ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config(args.n, args.nrhs), "impl": "reference",
            "cpu_baseline": {"value": v, "unit": "solves/s", "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": v, "unit": "solves/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    global LS
    LS = tuple(float(v) for v in args.ls.split(","))
    AUTO_RHO[0] = args.auto_rho
    if args.impl == "reference":
        return run_reference(args)
    import torch

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_2304_05460_gb300 import afn

    stream = torch.cuda.current_stream()
    if args.only:
        if args.only == "batched":
            out = run_batched(afn, args.batched, args.fp64_sample, stream)
        elif args.only == "clusters":
            out = run_clusters(afn, stream)
        elif args.only == "paper3d":
            prec = {"auto": afn.PREC_AUTO, "mixed": afn.PREC_MIXED, "df": afn.PREC_DF,
                    "fp64": afn.PREC_FP64}[args.paper_precision]
            out = run_paper3d(afn, stream, args.paper_kernel, args.paper_kmax, precision=prec,
                              kmode=args.paper_k, n=args.paper_n)
        else:
            out = run_serving(afn, args.serving, args.serving_rate, min(args.fp64_sample, 8))
        print(json.dumps({"only": args.only, args.only: out}), flush=True)
        return
    s = workload(args.n, args.nrhs)
    Xd = torch.tensor(s.X, device="cuda")
    Bd = torch.tensor(np.ascontiguousarray(s.B), device="cuda")

    precond_mode = [afn.PRECOND_AFN]   # the headline: AFN on every system

    def opts(profile, st=None):
        return afn.options(precision=afn.PREC_MIXED, rank_mode=afn.RANK_ESTIMATE,
                           rank_subsample=1000, seed=SEED, profile=profile,
                           stream=stream if st is None else st, max_iter=MAXIT,
                           precond=precond_mode[0])

    alg5_seen = []

    stats = {}
    iters_seen = []
    lock = threading.Lock()
    # the systems of a step are independent: by default each is built and solved on its own
    # stream from its own host thread, so the FP32-bound matvecs of one system overlap the
    # memory- and latency-bound apply and build kernels of the others
    streams = [torch.cuda.Stream() for _ in LS] if not args.sequential else []

    def one(l, profile, host, st):
        src_X, src_B = (s.X, s.B) if host else (Xd, Bd)
        h = afn.afn_build(src_X, afn.GAUSSIAN, l, MU, KMAX, W, opts(profile, st))
        x, info = afn.afn_solve(h, src_B, TOL)
        if info["converged"] != args.nrhs:
            raise RuntimeError("l=%g: %d/%d columns reached tol (relres max %.3e)"
                               % (l, info["converged"], args.nrhs, info["relres"].max()))
        with lock:
            if precond_mode[0] != afn.PRECOND_AFN:
                alg5_seen.append((l, "nystrom" if h.info.precond == afn.PRECOND_NYSTROM else "afn",
                                  int(h.info.k), int(info["iters"].max())))
                afn.afn_free(h)
                return
            iters_seen.append(int(info["iters"].max()))
            if profile:
                for nm in ("matvec32", "matvec64", "apply32", "fps", "knn", "chol", "trsm",
                           "fsai", "blas1", "rank"):
                    c, ms = afn.afn_get_kernel_stats(h, nm)
                    a = stats.setdefault(nm, [0, 0.0])
                    a[0] += c
                    a[1] += ms
        afn.afn_free(h)

    def step(profile, host=False):
        if args.sequential:
            for l in LS:
                one(l, profile, host, None)
            return
        errs = []

        def run(l, st):
            try:
                with torch.cuda.stream(st):
                    one(l, profile, host, st)
                st.synchronize()
            except BaseException as e:   # re-raised on the main thread
                errs.append(e)

        ts = [threading.Thread(target=run, args=(l, st)) for l, st in zip(LS, streams)]
        for t in ts:
            t.start()
        for t in ts:
            t.join()
        if errs:
            raise errs[0]

    for _ in range(args.warmup):
        step(0)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clk = Clocks(local)
    clk.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    launches0 = afn.afn_launch_count()
    e0.record(stream)
    for _ in range(args.steps):
        step(1)
    e1.record(stream)
    launches = afn.afn_launch_count() - launches0
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = clk.stop()
    ms = job_time_ms(e0.elapsed_time(e1), dist, "cuda")
    value = job_throughput(args.nrhs * len(LS) * args.steps, world, ms)

    # end to end through the C ABI with host buffers (copies inside the timed region)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        step(0, host=True)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e_val = args.nrhs * len(LS) * args.e2e_steps * world / e2e_s
    h2d = len(LS) * (s.X.nbytes + s.B.nbytes)
    d2h = len(LS) * s.B.nbytes

    # the paper's full scheme (Alg. 5): the same workload with the preconditioner chosen per
    # system by the Alg. 4 estimate (Nystrom below k = 2000, AFN above)
    alg5 = None
    if args.alg5_steps > 0:
        precond_mode[0] = afn.PRECOND_AUTO
        torch.cuda.synchronize()
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        for _ in range(args.alg5_steps):
            step(0)
        a1.record(stream)
        torch.cuda.synchronize()
        a_ms = job_time_ms(a0.elapsed_time(a1), dist, "cuda")
        precond_mode[0] = afn.PRECOND_AFN
        per = sorted(set(alg5_seen))
        alg5 = {"value": job_throughput(args.nrhs * len(LS) * args.alg5_steps, world, a_ms),
                "unit": "solves/s", "ms_per_step": a_ms / args.alg5_steps,
                "steps": args.alg5_steps,
                "systems": [{"l": l, "precond": pc, "k": k, "iters": it} for l, pc, k, it in per],
                "note": "Alg. 5: Nystrom preconditioner (eq. nystrom1-smw) when the Alg. 4 "
                        "estimate is below 2000, AFN otherwise; same schedule and tolerance"}

    # roofline of the dominant kernel (FP32 matvec): FP32-pipe bound, counted in FP32
    # lane operations per kernel-pair evaluation, 2d + 1 + nrhs (d subtractions, d
    # multiply-adds for r^2, the scale, and one multiply-add per right-hand side)
    mv_cnt, mv_ms = stats.get("matvec32", [0, 0.0])
    n = args.n
    nr_piece = min(args.nrhs, 32)
    ops_pair = 2 * D + 1 + nr_piece
    ops_per_launch = float(n) * n * ops_pair
    avg_ms = mv_ms / max(mv_cnt, 1)
    achieved = ops_per_launch / (avg_ms / 1e3) / 1e12 if mv_cnt else None
    peak = LANE_PEAK_TOPS
    roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tops/s",
            "frac": (achieved / peak) if achieved else None,
            "traffic": MATVEC32_TRAFFIC_BYTES if (n == N and nr_piece == 32) else None,
            "kernel": ("matvec32u_kernel<DS=8,NB=%d,Gaussian> (tcgen05)" % (nr_piece // 8)
                       if nr_piece >= 16 else "matvec32tca_kernel<DS=8,NB=%d,Gaussian>" % (nr_piece // 8)),
            "ops_per_pair": ops_pair,
            "pairs_per_launch": float(n) * n, "avg_launch_ms": avg_ms, "launches": mv_cnt,
            "peak_basis": "FP32 pipe: 152 SMs x 128 lanes x 2070 MHz, one lane operation per "
                          "lane per cycle (derived); ops = FP32 lane operations, 2d+1+nrhs per pair"}
    if achieved and nr_piece >= 16:
        # the contraction runs on the tensor cores; the FP32 pipe still evaluates every
        # kernel value: d subtractions, d FMAs and the split, 2d + 1 lane-operations a pair
        pairs_s = float(n) * n / (avg_ms / 1e3)
        eval_peak = N_SM * FP32_LANES * SM_MAX_MHZ * 1e6 / (2 * D + 1)
        roof["eval_bound"] = {"pairs_per_s": pairs_s, "peak_pairs_per_s": eval_peak,
                              "frac": pairs_s / eval_peak,
                              "basis": "FP32 pipe, 2d+1 lane-ops per kernel value (derived)"}
    if not args.sequential and mv_cnt:
        # the timed region runs the systems concurrently, so its launch durations include
        # the SMs shared with the other systems' kernels; the same matvec timed alone
        # (whole afn_kernel_matvec calls: p split, points, kernel, finish) for comparison
        torch.cuda.synchronize()
        for _ in range(2):
            afn.afn_kernel_matvec(Xd, afn.GAUSSIAN, 2.0, MU, Bd, precision=afn.PREC_MIXED,
                                  stream=stream)
        c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 10
        c0.record(stream)
        for _ in range(reps):
            afn.afn_kernel_matvec(Xd, afn.GAUSSIAN, 2.0, MU, Bd, precision=afn.PREC_MIXED,
                                  stream=stream)
        c1.record(stream)
        torch.cuda.synchronize()
        iso_ms = c0.elapsed_time(c1) / reps
        iso = ops_per_launch / (iso_ms / 1e3) / 1e12
        roof["isolated"] = {"avg_call_ms": iso_ms, "achieved": iso, "frac": iso / peak,
                            "basis": "afn_kernel_matvec alone, same points and 32 columns, "
                                     "CUDA events over %d calls" % reps}
        roof["note"] = ("timed-region launch durations include SMs shared with the "
                        "concurrently solved systems")
    kernels = {k: {"launches": v[0], "ms": round(v[1], 3)} for k, v in stats.items()}
    step_ms = ms / args.steps

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        t_cpu = time.perf_counter()
        v, detail, cores, _ = oracle_sample(args.n, args.nrhs, "baseline")
        t_cpu = time.perf_counter() - t_cpu
        cpu = {"value": v, "unit": "solves/s", "cores": cores, "kind": "oracle",
               "sample": "one bounded sample of %.1f s (measured): %s" % (t_cpu, detail)}

    fp64 = None
    if rank == 0 and not args.no_fp64:
        # plain FP64 GPU AFN-PCG on the l = 1 system, same RHS (the comparison arm)
        o64 = afn.options(precision=afn.PREC_FP64, rank_mode=afn.RANK_ESTIMATE,
                          rank_subsample=1000, seed=SEED, stream=stream, max_iter=MAXIT)
        torch.cuda.synchronize()
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        h = afn.afn_build(Xd, afn.GAUSSIAN, 1.0, MU, KMAX, W, o64)
        x, info = afn.afn_solve(h, Bd, TOL)
        f1.record(stream)
        torch.cuda.synchronize()
        fms = f0.elapsed_time(f1)
        fp64 = {"value": args.nrhs / (fms / 1e3), "unit": "solves/s", "system": "l=1",
                "ms": fms, "iters_max": int(info["iters"].max()),
                "converged": int(info["converged"])}
        afn.afn_free(h)

    # batched and serving: every rank solves the systems dealt to it (replicas)
    batched = None
    if args.batched > 0:
        try:
            batched = run_batched(afn, args.batched, args.fp64_sample, stream, rank, world, dist)
        except Exception as e:          # reported in the line, the headline stands
            batched = {"error": repr(e)}
    clusters = None
    if rank == 0 and args.clusters > 0:
        try:
            clusters = run_clusters(afn, stream)
        except Exception as e:
            clusters = {"error": repr(e)}
    one_rhs = None
    if rank == 0 and args.one_rhs > 0:
        try:
            one_rhs = run_one_rhs(afn, s, Xd, Bd, stream, opts)
        except Exception as e:
            one_rhs = {"error": repr(e)}
    serving = None
    if args.serving > 0:
        try:
            serving = run_serving(afn, args.serving, args.serving_rate, min(args.fp64_sample, 8),
                                  rank, world, dist)
        except Exception as e:
            serving = {"error": repr(e)}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": step_ms,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f32+f64", "data": "synthetic", "config": config(args.n, args.nrhs),
                "schedule": ("sequential: the systems of a step one after another"
                             if args.sequential else
                             "concurrent: each system of a step built and solved on its own "
                             "stream and host thread"),
                "e2e": {"value": e2e_val, "unit": "solves/s", "h2d_bytes_per_step": h2d,
                        "d2h_bytes_per_step": d2h},
                "gpu_launches": launches, "roofline": roof, "cpu_baseline": cpu, "clocks": clocks,
                "alg5": alg5,
                "kernels": kernels,
                "kernels_note": ("per-class device time summed over launches (CUDA events); "
                                 "with the concurrent schedule the classes of different "
                                 "systems overlap, so the sums exceed the step time"
                                 if not args.sequential else
                                 "per-class device time summed over launches (CUDA events)"),
                "fp64_gpu": fp64,
                "pcg_iters_max": iters_seen[-len(LS):] if iters_seen else None,
                "batched": batched, "serving": serving, "clusters_3d": clusters,
                "normal_8d_1rhs": one_rhs,
                "autotuner": afn.afn_tune_entries()}
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
