"""Stored expected values (tests/golden/oracle_golden.json, written by
tests/golden/make_golden.py from the FP64 oracle alone, each with the passage it
restates): the oracle must still reproduce them (CPU), and the library's
integer results must equal them (GPU, no oracle at run time)."""
import json
import os

import numpy as np
import pytest

import oracle
from paper_2304_05460_gb300 import inputs

GOLDEN = json.load(open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                                     "oracle_golden.json")))


def test_oracle_reproduces_golden():
    g = GOLDEN
    X = inputs.uniform_points(96, 3, 2024)
    assert oracle.fps(X, g["fps"]["k"], g["fps"]["start"]).tolist() == g["fps"]["idx"]
    pat, _ = oracle.knn_pattern(inputs.normal_points(40, 2, 2025), g["knn"]["w"])
    assert pat.astype(int).tolist() == g["knn"]["pattern"]
    r = g["rank"]
    got = oracle.rank_estimate(inputs.uniform_points(400, 3, 2026), oracle.GAUSSIAN, r["l"], r["mu"],
                               m=r["m"], seed=r["seed"], k_max=r["k_max"])
    assert got == (r["k"], r["r"], r["branch"])
    s = inputs.uniform_cube_3d()
    f = oracle.afn_build(s.X, s.kernel, s.l, s.mu, s.k, s.w)
    _, it, rel, st = oracle.pcg(f, s.B[:, 0], 1e-6, max_iter=500)
    assert (it, st) == (g["pcg_uniform_cube"]["iters"], g["pcg_uniform_cube"]["status"])
    assert rel <= 1e-6
    nys = g["nystrom_apply"]
    fn = oracle.nystrom_build(inputs.uniform_points(150, 2, 2027), oracle.GAUSSIAN, 0.25, 1e-2, 30)
    sv = oracle.nystrom_apply(fn, inputs.rhs(150, 1, 2028)[:, 0])
    assert np.allclose(sv[:8], nys["s_head"], rtol=nys["rtol"], atol=0)


@pytest.fixture(scope="module")
def afn():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2304_05460_gb300 import afn as a
    return a


@pytest.mark.gpu
def test_library_matches_golden(afn):
    g = GOLDEN
    X = inputs.uniform_points(96, 3, 2024)
    assert afn.afn_fps(X, g["fps"]["k"], g["fps"]["start"]).tolist() == g["fps"]["idx"]
    pat = afn.afn_knn_pattern(inputs.normal_points(40, 2, 2025), g["knn"]["w"])
    assert pat.astype(int).tolist() == g["knn"]["pattern"]
    s = inputs.uniform_cube_3d()
    h = afn.afn_build(s.X, s.kernel, s.l, s.mu, s.k, s.w, precision=afn.PREC_FP64)
    x, info = afn.afn_solve(h, s.B, 1e-6)
    assert info["converged"] == 1
    assert abs(int(info["iters"][0]) - g["pcg_uniform_cube"]["iters"]) <= 2
    afn.afn_free(h)
