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


def test_algorithmic_bytes_formula():
    """Encoder, block-build and sort bytes of the stage rooflines, on a
    hand-sized table: 3 rows, a string column of 4, 5 and 0 bytes read by a
    Jaccard (q = 3) predicate and an int32 key."""
    import bench
    import synth
    t = synth.table_from_rows(["s", "k"], ["string", "int32"], [("abcd", 1), ("abcde", 2), ("", 1)])
    mds = [[synth.eq(1), synth.jac(0, 1, 2)]]
    got = bench.algorithmic_bytes(t, mds, {"emitted_pairs": 5})
    read = 9 + 4 * 4 + 3 * 4                 # string bytes + offsets, int32 keys
    grams = 2 + 3 + 0                        # |s| - 2 grams per string
    assert got["encode"] == read + 4 * 3 * 1 + 4 * grams + 4 * 4
    assert got["block_build"] == 4 * 3 * 1 + 4 * 3
    assert got["sort"] == 2 * 8 * 5 * 1      # 2 bits per row id, two ids: one 8-bit pass


class _Info:
    def __init__(self, prog):
        self.op_pred = prog + [0] * (128 - len(prog))
        self.n_ops = len(prog)


def test_plan_units_only_for_the_plan_they_were_counted_for():
    import json
    import os
    import bench
    path = os.path.join(bench.GOLDEN, "plan_units_c2.json")
    if not os.path.exists(path):
        assert bench.plan_units(_Info([2, 8]), 4) is None
        return
    d = json.load(open(path))
    assert bench.plan_units(_Info(list(d["program_ids"])), 4)["units"]["total"] == d["units"]["total"]
    assert bench.plan_units(_Info(list(reversed(d["program_ids"]))), 4) is None
