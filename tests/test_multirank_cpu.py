"""The N>1 path of bench.py on CPU: replicas on a world-size-2 gloo group. Each rank reports
its own work and device time; the job's throughput is all ranks' work over the slowest rank's
time, and every rank agrees on it."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    # rank r did (r+1) * 1e9 units in (r+1) * 0.5 s
    value, t_max = bench.aggregate_over_ranks((rank + 1) * 0.5, (rank + 1) * 1e9, dist)
    q.put((rank, value, t_max))
    dist.destroy_process_group()


def test_replica_aggregation_on_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    out = sorted(q.get(timeout=10) for _ in range(2))
    for rank, value, t_max in out:
        assert t_max == pytest.approx(1.0)          # slowest rank
        assert value == pytest.approx(3e9 / 1.0)    # all units over the slowest time


def test_single_process_aggregation_is_plain_ratio():
    import bench

    v, t = bench.aggregate_over_ranks(2.0, 5e9, None)
    assert t == 2.0 and v == pytest.approx(2.5e9)
