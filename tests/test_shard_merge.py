"""Sharded evaluation, host side: the library's k-way merge of sorted pair
lists (hb_merge_pairs) and the final gather of a sharded run, with the ranks
as two gloo processes on the CPU.  Each rank keeps the oracle's pairs of the
blocks it owns (the owner rank of include/hb.h's hb_set_shard); the gathered
and merged lists must be disjoint and give the oracle's whole result."""
import ctypes
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2410_04349_gb300 import hb

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _sorted(p):
    p = np.asarray(p, np.int64).reshape(-1, 2)
    return p[np.lexsort((p[:, 1], p[:, 0]))]


def test_merge_gives_the_sorted_union():
    rng = np.random.default_rng(7)
    for k in (1, 2, 3, 7):
        lists = []
        for _ in range(k):
            n = int(rng.integers(0, 300))
            lists.append(_sorted(rng.integers(0, 50, size=(n, 2))))
        got = hb.merge_pairs(lists)
        want = _sorted(np.concatenate(lists) if lists else np.zeros((0, 2)))
        assert np.array_equal(got, want)
    assert hb.merge_pairs([]).shape == (0, 2)
    assert np.array_equal(hb.merge_pairs([np.zeros((0, 2)), np.array([[1, 2]])]), [[1, 2]])


def test_merge_rejects_bad_arguments():
    L = hb.lib()
    one = np.array([[1, 2]], np.uint32)
    ptrs = (ctypes.c_void_p * 1)(one.ctypes.data)
    out = np.zeros((1, 2), np.uint32)
    bad = np.array([-1], np.int64)
    assert L.hb_merge_pairs(ptrs, bad.ctypes.data, 1, out.ctypes.data) == hb.HB_ERR_ARG
    cnt = np.array([1], np.int64)
    assert L.hb_merge_pairs(None, cnt.ctypes.data, 1, out.ctypes.data) == hb.HB_ERR_ARG
    assert L.hb_merge_pairs(ptrs, cnt.ctypes.data, 1, None) == hb.HB_ERR_ARG
    assert L.hb_merge_pairs(ptrs, cnt.ctypes.data, -1, out.ctypes.data) == hb.HB_ERR_ARG
    assert L.hb_merge_pairs(None, None, 0, None) == hb.HB_OK


def test_owner_rank_spreads_blocks_over_the_ranks():
    from shard_helpers import fmix32, shard_of
    # the finaliser is a bijection of 32-bit words (xor-shifts and odd multipliers)
    xs = np.arange(200_000, dtype=np.int64)
    assert len({fmix32(int(x)) for x in xs}) == len(xs)
    assert fmix32(0) == 0
    # every rank gets a fair share of 3000 (md, row) block identities
    counts = np.bincount([shard_of(md, row, 3) for md in range(3) for row in range(1000)], minlength=3)
    assert counts.min() > 800


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import sys
    sys.path[:0] = [ROOT, os.path.join(ROOT, "tests")]
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle
    import synth
    from paper_2410_04349_gb300 import hb as hbm
    from shard_helpers import expected_shards
    t, mds = synth.config1(n=600)
    full, _ = oracle.block_hash(t, mds, threads=1)
    mine = full[expected_shards(t, mds, full, world) == rank]
    gathered = [None] * world
    dist.all_gather_object(gathered, mine)
    merged = hbm.merge_pairs(gathered)
    q.put((rank, len(mine), bool(np.array_equal(merged, full)), int(sum(len(g) for g in gathered)), len(full)))
    dist.destroy_process_group()


def test_two_gloo_ranks_gather_and_merge_their_shards():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get() for _ in range(2))
    for rank, n_mine, equal, total, n_full in res:
        assert equal, f"rank {rank}: merged shards differ from the whole result"
        assert total == n_full   # disjoint shards: their sizes add up to the whole
    assert all(n > 0 for _, n, _, _, _ in res), "one rank owned no pair of this table"
