"""GPU tests of the serving loop: every result reaches tol (oracle FP64
residual), a request's result is bit-identical alone and in a mix of
requests that arrive while it runs (and equal to the batched solve of the
same system), admission respects the device-memory budget, and a failing
request reports its error without disturbing the others."""
import time

import numpy as np
import pytest

import oracle
from paper_2304_05460_gb300 import inputs

pytestmark = pytest.mark.gpu

G, M32 = 0, 1


@pytest.fixture(scope="module")
def afn():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2304_05460_gb300 import afn as a
    return a


def request(i, n=None):
    """A small request of the serving workload's kind (d in {3, 8, 16},
    Gaussian or Matern, l = median distance x log-uniform [0.1, 10] drawn
    as for the stream, 1..16 RHS)."""
    g = inputs.rng(5000 + i)
    n = n or int(np.exp(g.uniform(np.log(300), np.log(2500))))
    d = int(g.choice([3, 8, 16]))
    ker = int(g.integers(0, 2))
    nrhs = int(g.integers(1, 17))
    X = g.standard_normal((n, d))
    B = np.asfortranarray(g.standard_normal((nrhs, n)).T)
    l = inputs.median_pairwise_distance(X, 5000 + i) * float(np.exp(g.uniform(np.log(0.3), np.log(3.0))))
    mu = float(np.exp(g.uniform(np.log(1e-3), np.log(1e-1))))
    return dict(points=X, kernel=ker, l=l, mu=mu, k_max=min(n // 4, 1000), fsai_nnz=32), B


def drain(srv, ids, timeout=300.0):
    out = {}
    t0 = time.time()
    while len(out) < len(ids):
        for rid in srv.poll(wait_ms=200):
            out[rid] = srv.result(rid)
        assert time.time() - t0 < timeout, "server did not finish"
    return out


def relres(sy, x, B):
    X = sy["points"]
    r = oracle.true_relres(X, sy["kernel"], sy["l"], sy["mu"], np.asarray(x).reshape(X.shape[0], -1), B)
    return np.where(np.linalg.norm(B, axis=0) > 0, r, 0.0)


def test_server_requests_reach_tol(afn):
    reqs = [request(i) for i in range(12)]
    srv = afn.Server(seed=3, max_iter=2000)
    ids = [srv.submit(sy, B, 1e-6) for sy, B in reqs]
    res = drain(srv, ids)
    st = srv.stats()
    srv.close()
    assert st["completed"] == 12 and st["active"] == 0 and st["reserved_bytes"] == 0
    for rid, (sy, B) in zip(ids, reqs):
        x, info = res[rid]
        assert info["status"] == afn.AFN_OK and info["converged"] == B.shape[1]
        assert relres(sy, x, B).max() <= 1e-6
        assert info["latency_ms"] >= info["solve_ms"] >= 0.0


def test_alone_and_in_mix_bit_identical(afn):
    sy, B = request(100, n=1800)
    srv = afn.Server(seed=3, max_iter=2000)
    rid = srv.submit(sy, B, 1e-6)
    x_alone, _ = drain(srv, [rid])[rid]
    srv.close()
    # the same request arriving while others are building and solving
    others = [request(200 + i) for i in range(10)]
    srv = afn.Server(seed=3, max_iter=2000, build_threads=4)
    ids = [srv.submit(s, b, 1e-6) for s, b in others[:6]]
    time.sleep(0.05)
    rid = srv.submit(sy, B, 1e-6)
    ids += [srv.submit(s, b, 1e-6) for s, b in others[6:]]
    res = drain(srv, ids + [rid])
    srv.close()
    x_mix, info = res[rid]
    assert info["status"] == afn.AFN_OK
    assert np.array_equal(x_alone, x_mix)
    # and the batched solve of the same system runs the same arithmetic
    b = afn.afn_build_batched([sy], seed=3, max_iter=2000)
    xb, _ = afn.afn_solve_batched(b, [B], 1e-6)
    assert np.array_equal(np.asarray(xb[0]).reshape(x_mix.shape), x_mix)


def test_admission_by_memory_budget(afn):
    reqs = [request(300 + i) for i in range(8)]
    # a budget that admits only a couple of these requests at a time
    budget = 60 << 20
    srv = afn.Server(memory_budget=budget, seed=3, max_iter=2000, build_threads=4)
    ids = [srv.submit(sy, B, 1e-6) for sy, B in reqs]
    res = drain(srv, ids)
    st = srv.stats()
    srv.close()
    sizes = [res[r][1]["device_bytes"] for r in ids]
    assert st["peak_reserved_bytes"] <= max(budget, max(sizes))
    assert st["completed"] == 8
    for rid, (sy, B) in zip(ids, reqs):
        assert relres(sy, res[rid][0], B).max() <= 1e-6


def test_failing_request_reports_error(afn):
    good, Bg = request(400)
    bad, Bb = request(401)
    bad = dict(bad, mu=-1.0)
    srv = afn.Server(seed=3)
    i_bad = srv.submit(bad, Bb, 1e-6)
    i_good = srv.submit(good, Bg, 1e-6)
    done = {}
    t0 = time.time()
    while len(done) < 2 and time.time() - t0 < 120:
        for rid in srv.poll(wait_ms=200):
            done[rid] = True
    with pytest.raises(afn.AfnError) as e:
        srv.result(i_bad)
    assert e.value.status == afn.AFN_ERR_ARG
    x, info = srv.result(i_good)
    srv.close()
    assert info["status"] == afn.AFN_OK
    assert relres(good, x, Bg).max() <= 1e-6


def test_submit_rejects_nan(afn):
    sy, B = request(500)
    B[0, 0] = np.nan
    srv = afn.Server()
    with pytest.raises(afn.AfnError) as e:
        srv.submit(sy, B, 1e-6)
    srv.close()
    assert e.value.status == afn.AFN_ERR_ARG
