"""Multi-process host logic of bench.py on CPU (gloo, world size 2): the
batched and serving workloads and single systems run as independent
replicas, one per GPU, so the only cross-rank step is the job time = the
maximum of the ranks' timed regions, and the throughput counts every rank's
solves over it."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local = [120.0, 250.0][rank]
    ms = bench.job_time_ms(local, dist, "cpu")
    thr = bench.job_throughput(128, world, ms)
    # the batched/serving replicas: this rank's share of the dealt systems, the
    # summed counts and the gathered latencies
    costs = [float(n) ** 2 for n in (300, 8000, 900, 4100, 256, 5000, 7000, 1200)]
    share = bench.deal(costs, world)[rank]
    cols = bench.job_sum(8 * len(share), dist, "cpu")
    lat = bench.job_gather([float(rank * 100 + i) for i in share], dist)
    q.put((rank, ms, thr, share, cols, lat))
    dist.destroy_process_group()


def test_replica_job_time_is_max_over_ranks():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    out = [q.get(timeout=120) for _ in ps]
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    shares = {}
    for rank, ms, thr, share, cols, lat in out:
        assert ms == 250.0
        assert thr == pytest.approx(128 * 2 / 0.25)
        shares[rank] = share
        assert cols == 8 * 8                      # every system's columns counted once
        assert len(lat) == 8
    assert sorted(shares[0] + shares[1]) == list(range(8))   # each system on exactly one rank
    assert set(shares[0]).isdisjoint(shares[1])


def test_deal_balances_cost_and_is_deterministic():
    sys.path.insert(0, ROOT)
    import bench
    costs = [float(n) ** 2 for n in [8192, 256, 300, 5000, 4000, 4000, 1000, 7000, 2500, 600]]
    for world in (1, 2, 3, 4):
        sh = bench.deal(costs, world)
        assert sh == bench.deal(costs, world)
        assert sorted(i for s in sh for i in s) == list(range(len(costs)))
        loads = [sum(costs[i] for i in s) for s in sh]
        # longest-first greedy: no rank exceeds the mean by more than the largest item
        assert max(loads) <= sum(costs) / world + max(costs)
    assert bench.deal(costs, 1) == [list(range(len(costs)))]


def test_single_process_time_is_local():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.job_time_ms(42.0, None, "cpu") == 42.0
    assert bench.job_throughput(10, 1, 500.0) == pytest.approx(20.0)

