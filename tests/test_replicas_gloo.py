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
    q.put((rank, ms, thr))
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
    for rank, ms, thr in out:
        assert ms == 250.0
        assert thr == pytest.approx(128 * 2 / 0.25)


def test_single_process_time_is_local():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.job_time_ms(42.0, None, "cpu") == 42.0
    assert bench.job_throughput(10, 1, 500.0) == pytest.approx(20.0)
