"""bench.py's whole-job aggregation across ranks (sum of units, slowest
rank's time), run as two gloo processes on the CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    units, secs = bench.aggregate(100.0 * (rank + 1), 1.0 + rank, world)
    q.put((rank, units, secs))
    dist.destroy_process_group()


def test_aggregate_two_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(60)
        assert p.exitcode == 0
    res = sorted(q.get() for _ in range(2))
    for _, units, secs in res:
        assert units == 300.0 and secs == 2.0


def test_aggregate_single_rank_is_identity():
    import bench
    assert bench.aggregate(5.0, 2.0, 1) == (5.0, 2.0)


def test_algorithmic_ops_formula():
    import bench
    logs = [{"kind": 2, "evaluated": 10, "stage1": 4, "stage2": 1, "core": 50},
            {"kind": 4, "evaluated": 7, "stage1": 0, "stage2": 0, "core": 0}]
    got = bench.algorithmic_ops(logs, examined=100, n_eq=3)
    assert got == 100 * (3 * 3 + 3) + 10 * 4 + 4 * 18 + 50 * 5 + 7 * 3
