"""Sharded evaluation on the GPU (hb_set_shard): the ranks run one after the
other on one GPU, as separate processes would on theirs.  Each rank's pairs
are exactly the pairs of the blocks the owner function gives it (computed
here from the data, tests/shard_helpers.py), the ranks' outputs are disjoint,
and merged (hb_merge_pairs) they equal the unsharded result and the oracle's."""
import numpy as np
import pytest

import oracle
import synth
from paper_2410_04349_gb300 import hb
from shard_helpers import expected_shards

pytestmark = pytest.mark.gpu


def _run(t, mds, rank, world):
    with hb.Context(device=0) as ctx:
        ctx.load_table(0, t.n_rows, t.columns)
        for md in mds:
            ctx.add_md(md)
        ctx.set_shard(rank, world)
        ctx.plan("rule_data")
        pairs = ctx.block()
        st = ctx.stats()
    return pairs, st


@pytest.mark.parametrize("world", [2, 3])
def test_shards_are_the_owned_blocks_and_merge_to_the_whole(world):
    t, mds = synth.config1(n=2000)
    full, cand = oracle.block_hash(t, mds)
    whole, st1 = _run(t, mds, 0, 1)
    assert np.array_equal(whole, full)
    want = expected_shards(t, mds, full, world)
    parts, cands = [], 0
    for r in range(world):
        p, st = _run(t, mds, r, world)
        assert np.array_equal(p, full[want == r]), f"rank {r} of {world}"
        parts.append(p)
        cands += st["candidate_pairs"]
    assert np.array_equal(hb.merge_pairs(parts), full)
    assert sum(len(p) for p in parts) == len(full)
    assert cands == st1["candidate_pairs"]   # every candidate evaluated by exactly one rank


def test_shards_on_the_benchmark_shape():
    # 20,000 tuples of the 8-attribute schema with its four rules (keys of 1-3
    # columns, Zipf-sized groups, packed small blocks)
    t, mds = synth.config2(n=20_000)
    whole, _ = _run(t, mds, 0, 1)
    parts = [_run(t, mds, r, 4)[0] for r in range(4)]
    assert np.array_equal(hb.merge_pairs(parts), whole)
    assert sum(len(p) for p in parts) == len(whole)
    assert sum(1 for p in parts if len(p)) >= 2


def test_stream_and_batch_refuse_a_shard():
    t, mds = synth.config1(n=200)
    with hb.Context(device=0) as ctx:
        ctx.load_table(0, t.n_rows, t.columns)
        for md in mds:
            ctx.add_md(md)
        ctx.set_shard(1, 2)
        with pytest.raises(hb.HBError) as e:
            ctx.block_batch(np.array([0, 100, 200], np.int64))
        assert e.value.status == hb.HB_ERR_STATE
        with pytest.raises(hb.HBError) as e:
            ctx.block_stream(t.n_rows, t.columns)
        assert e.value.status == hb.HB_ERR_STATE
        with pytest.raises(hb.HBError) as e:
            ctx.set_shard(2, 2)
        assert e.value.status == hb.HB_ERR_ARG
