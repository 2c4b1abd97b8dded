"""Multi-process path of bench.py on CPU (gloo, world size 2): each rank solves its own replica,
the job time is the slowest rank's, the rate counts every rank's units.  No data-path
collective exists (replicas only); this checks the timing aggregation the bench relies on."""
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    import sys
    import torch.distributed as dist
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    slowest = bench.max_over_ranks(10.0 * (rank + 1), world, device="cpu")
    q.put((rank, slowest, bench.throughput(5, world, slowest)))
    dist.barrier()
    dist.destroy_process_group()


def test_gloo_world2_max_over_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    assert [g[1] for g in got] == [20.0, 20.0]
    assert got[0][2] == pytest.approx(2 * 5 / 0.020)


def test_single_rank_helpers():
    import bench
    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.throughput(10, 1, 500.0) == pytest.approx(20.0)
