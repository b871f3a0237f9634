"""Writes tests/golden/oracle_golden.json: expected values computed by the FP64
oracle (and nothing else) on seeded synthetic inputs, each with the passage of
the paper it restates.  Run from the repository root:

    python tests/golden/make_golden.py

The CPU tests check that the oracle still reproduces every value (an oracle
change that moves one must name the passage that justifies it); the GPU tests
compare the library's integer results with them directly.
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2304_05460_gb300 import inputs  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_golden.json")


def main():
    g = {}
    # FPS (Alg. 6): order of 24 landmarks among 96 uniform points in the unit cube, start 0
    X = inputs.uniform_points(96, 3, 2024)
    g["fps"] = {"cite": "Alg. 6 (farthest point sampling)", "input": "uniform_points(96, 3, 2024)",
                "k": 24, "start": 0, "idx": [int(v) for v in oracle.fps(X, 24, 0)]}
    # KNN pattern (Sec. 3.1): w - 1 nearest lower-numbered points, then the point itself
    Xr = inputs.normal_points(40, 2, 2025)
    pat, _ = oracle.knn_pattern(Xr, 6)
    g["knn"] = {"cite": "Sec. 3.1 (FSAI sparsity pattern)", "input": "normal_points(40, 2, 2025)",
                "w": 6, "pattern": pat.astype(int).tolist()}
    # Alg. 4 on 400 uniform points, m = 120, seed 9
    Xa = inputs.uniform_points(400, 3, 2026)
    k, r, br = oracle.rank_estimate(Xa, oracle.GAUSSIAN, 0.2, 1e-2, m=120, seed=9, k_max=400)
    g["rank"] = {"cite": "Alg. 4 (Nystrom rank estimate)", "input": "uniform_points(400, 3, 2026)",
                 "l": 0.2, "mu": 1e-2, "m": 120, "seed": 9, "k_max": 400, "k": k, "r": r,
                 "branch": br}
    # the n = 2000 uniform-cube workload, FP64 AFN-PCG (Alg. 2, Alg. 3, PCG to 1e-6)
    s = inputs.uniform_cube_3d()
    f = oracle.afn_build(s.X, s.kernel, s.l, s.mu, s.k, s.w)
    x, it, rel, st = oracle.pcg(f, s.B[:, 0], 1e-6, max_iter=500)
    g["pcg_uniform_cube"] = {"cite": "Alg. 2, Alg. 3 and PCG (Sec. 5 stopping rule)",
                             "input": "uniform_cube_3d()", "tol": 1e-6, "iters": it,
                             "status": st, "relres_bound": 1e-6}
    # Nystrom apply, eq. (nystrom1-smw): first 8 entries of s = M^{-1} r (permuted order)
    Xn = inputs.uniform_points(150, 2, 2027)
    fn = oracle.nystrom_build(Xn, oracle.GAUSSIAN, 0.25, 1e-2, 30)
    rv = inputs.rhs(150, 1, 2028)[:, 0]
    sv = oracle.nystrom_apply(fn, rv)
    g["nystrom_apply"] = {"cite": "Sec. 2, eq. (nystrom1-smw)", "input": "uniform_points(150, 2, 2027), "
                          "rhs(150, 1, 2028), l = 0.25, mu = 1e-2, k = 30",
                          "s_head": [float(v) for v in sv[:8]], "rtol": 1e-12}
    with open(OUT, "w") as fh:
        json.dump(g, fh, indent=1)
        fh.write("\n")
    print("wrote", OUT)


if __name__ == "__main__":
    main()
