"""GPU parity of root-edge hash partitioning (Section 5.3, "Data
partitioning", hb_set_partitions): for every number of partitions the pair set
equals the oracle's plain blocking result, the candidate count equals the
partition oracle's, and the branches are the oracle's root edges."""
import numpy as np
import pytest

import oracle
import oracle.partition as op
import synth
from paper_2410_04349_gb300 import hb

pytestmark = pytest.mark.gpu

RULES = {
    "int_and_string_roots": [[synth.eq(2), synth.ed(0, 3)], [synth.eq(3), synth.jac(1, 1, 3)],
                             [synth.eq(2), synth.eq(3), synth.absdiff(4, 0.5)]],
    "prefix_root": [[synth.eq_prefix(0, 2), synth.ed(0, 2)], [synth.eq(2), synth.jac(1, 1, 2)]],
    "with_all_tuples_branch": [[synth.eq(3), synth.ed(0, 2)], [synth.ed(0, 1), synth.absdiff(4, 0.1)]],
    "equality_only": [[synth.eq(2), synth.eq(3)], [synth.eq(3), synth.ed(1, 4)]],
}


def _run(R, mds, m, S=None, mode="given"):
    with hb.Context(device=0) as ctx:
        ctx.load_table(0, R.n_rows, R.columns)
        if S is not None:
            ctx.load_table(1, S.n_rows, S.columns)
        for md in mds:
            ctx.add_md(md)
        ctx.set_partitions(m)
        info = ctx.plan(mode)
        pairs = ctx.block()
        st = ctx.stats()
    return pairs, st, info


def _branch_preds(mds, self_join=True):
    """The oracle's branches as distinct-predicate ids (-1: the all-tuples branch)."""
    dp = [oracle._norm_pred(p) for p in oracle.distinct_predicates(mds)]
    out = []
    for md, key in zip(mds, op.root_keys(mds, self_join)):
        if key is None:
            pid = -1
        else:
            pid = next(dp.index(oracle._norm_pred(p)) for p in md
                       if p[0] in ("eq", "eq_prefix") and (not self_join or p[1] == p[2]))
        if pid not in out:
            out.append(pid)
    return out


@pytest.mark.parametrize("rules", sorted(RULES))
@pytest.mark.parametrize("m", [1, 3, 64, 1 << 20])
def test_self_join_partitions(rules, m):
    t = synth.random_small(21, n=700, null_rate=0.05)
    mds = RULES[rules]
    want, _ = oracle.block_hash(t, mds)
    pairs, st, info = _run(t, mds, m)
    assert np.array_equal(pairs, want)
    assert st["candidate_pairs"] == op.candidates(t, mds, m)
    assert list(info.branch_pred[:info.n_branches]) == _branch_preds(mds)


@pytest.mark.parametrize("m", [2, 97])
def test_cross_relation_partitions(m):
    R = synth.random_small(31, n=400, null_rate=0.1)
    S = synth.random_small(32, n=500, null_rate=0.1)
    mds = [[synth.eq_prefix(0, 1), synth.ed(0, 2)], [synth.eq(2), synth.eq(3), synth.jac(1, 1, 3)]]
    want, _ = oracle.block_hash(R, mds, S=S)
    pairs, st, info = _run(R, mds, m, S=S)
    assert np.array_equal(pairs, want)
    assert st["candidate_pairs"] == op.candidates(R, mds, m, S=S)
    assert list(info.branch_pred[:info.n_branches]) == _branch_preds(mds, self_join=False)


def test_benchmark_rules_every_plan_mode():
    t, mds = synth.config2(n=3000, cards=(30, 100, 300))
    want, _ = oracle.block_hash(t, mds)
    cand = op.candidates(t, mds, 256)
    for mode in ("given", "rule_data", "random"):
        pairs, st, _ = _run(t, mds, 256, mode=mode)
        assert np.array_equal(pairs, want), mode
        assert st["candidate_pairs"] == cand, mode


def test_switching_back_restores_exact_groups():
    t = synth.random_small(41, n=500, null_rate=0.05)
    mds = RULES["int_and_string_roots"]
    want, cand = oracle.block_hash(t, mds)
    with hb.Context(device=0) as ctx:
        ctx.load_table(0, t.n_rows, t.columns)
        for md in mds:
            ctx.add_md(md)
        ctx.set_partitions(8)
        ctx.plan("given")
        p8 = ctx.block()
        c8 = ctx.stats()["candidate_pairs"]
        ctx.set_partitions(0)
        p0 = ctx.block()       # plans again with exact groups
        c0 = ctx.stats()["candidate_pairs"]
    assert np.array_equal(p8, want) and np.array_equal(p0, want)
    assert c8 == op.candidates(t, mds, 8)
    assert c0 == cand


def test_partitioned_streaming_and_batches_are_refused():
    R = synth.random_small(51, n=200)
    mds = RULES["prefix_root"]
    with hb.Context(device=0) as ctx:
        ctx.load_table(0, R.n_rows, R.columns)
        for md in mds:
            ctx.add_md(md)
        ctx.set_partitions(4)
        with pytest.raises(hb.HBError) as e:
            ctx.block_stream(R.n_rows, R.columns)
        assert e.value.status == hb.HB_ERR_STATE
    t = synth.config4(n_jobs=5, sizes=[30, 40, 50, 60, 70])[0]
    with hb.Context(device=0) as ctx:
        ctx.load_table(0, t.n_rows, t.columns)
        ctx.add_md([synth.eq(2), synth.ed(0, 2)])
        ctx.set_partitions(4)
        with pytest.raises(hb.HBError) as e:
            ctx.block_batch(t.job_offsets)
        assert e.value.status == hb.HB_ERR_STATE
