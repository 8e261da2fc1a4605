"""Parity at the benchmark's full sizes, in the launch configuration bench.py
times: every sampled emitted pair is checked by the oracle, sampled blocks
are recomputed in full by the oracle's nested loop, and sampled candidate
pairs that were not emitted are confirmed as non-witnessed."""
import numpy as np
import pytest

import oracle
import synth
from paper_2410_04349_gb300 import hb

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


def _block_rows(t, md, rng, max_rows=1500, n_blocks=4):
    """Row sets of a few random groups of one MD's equality keys (the oracle
    recomputes each group in full)."""
    keys = []
    for p in md:
        if p[0] not in ("eq", "eq_prefix"):
            continue
        c = t.columns[p[1]]
        if c.type == "string":
            o = c.offsets.astype(np.int64)
            k = p[3] if p[0] == "eq_prefix" else None
            vals = [bytes(c.data[o[i]:o[i + 1]])[:k] if k else bytes(c.data[o[i]:o[i + 1]]) for i in range(t.n_rows)]
            keys.append(np.array([hash(v) for v in vals], np.int64))
        else:
            keys.append(c.data.astype(np.int64))
    kk = np.stack(keys, axis=1)
    _, inv, cnt = np.unique(kk, axis=0, return_inverse=True, return_counts=True)
    inv = inv.ravel()
    ok = np.nonzero((cnt >= 2) & (cnt <= max_rows))[0]
    picks = rng.choice(ok, size=min(n_blocks, len(ok)), replace=False)
    big = np.argmax(np.where(cnt <= max_rows, cnt, 0))
    picks = np.unique(np.concatenate([picks, [big]]))
    return [np.nonzero(inv == g)[0] for g in picks]


def _check(t, mds, pairs, rng, S=None):
    # 1. sampled emitted pairs satisfy the disjunction
    idx = rng.choice(len(pairs), size=min(20000, len(pairs)), replace=False)
    assert oracle.check_pairs(t, mds, pairs[idx], S=S).all()
    if S is not None:
        return
    emitted = set(map(tuple, pairs.tolist()))
    # 2. whole blocks recomputed by the nested loop
    for md in mds:
        for rows in _block_rows(t, md, rng):
            want = oracle.block_literal(t.take(rows), mds)
            want_g = {(int(min(rows[i], rows[j])), int(max(rows[i], rows[j]))) for i, j in want.tolist()}
            rs = set(rows.tolist())
            got = {p for p in emitted if p[0] in rs and p[1] in rs}
            assert got == want_g
            # 3. non-emitted pairs of the block are confirmed negative
            neg = [(int(min(a, b)), int(max(a, b))) for a, b in rng.choice(rows, size=(200, 2))
                   if a != b and (min(a, b), max(a, b)) not in emitted]
            if neg:
                assert not oracle.check_pairs(t, mds, np.array(neg)).any()


def test_config2_full_size():
    t, mds = synth.config2()
    with hb.Context(device=0) as ctx:
        ctx.load_table(0, t.n_rows, t.columns)
        for md in mds:
            ctx.add_md(md)
        ctx.plan("rule_data")
        pairs = ctx.block()
        st = ctx.stats()
    assert st["candidate_pairs"] > 1e9 and len(pairs) > 50000
    assert np.all(pairs[:-1, 0] <= pairs[1:, 0]) and np.all(pairs[:, 0] < pairs[:, 1])
    _check(t, mds, pairs, np.random.default_rng(1))


def test_config3_full_size_streamed():
    r, s, mds = synth.config3()
    with hb.Context(device=0) as ctx:
        ctx.load_table(0, r.n_rows, r.columns)
        for md in mds:
            ctx.add_md(md)
        pairs = ctx.block_stream(s.n_rows, s.columns)
    assert len(pairs) > 10000
    _check(r, mds, pairs, np.random.default_rng(2), S=s)


def test_config4_full_size_batched():
    t, mds = synth.config4()
    with hb.Context(device=0) as ctx:
        ctx.load_table(0, t.n_rows, t.columns)
        for md in mds:
            ctx.add_md(md)
        pairs, offs = ctx.block_batch(t.job_offsets)
    rng = np.random.default_rng(3)
    jobs = rng.choice(len(t.job_offsets) - 1, size=40, replace=False)
    for j in jobs:
        a, b = t.job_offsets[j], t.job_offsets[j + 1]
        if b - a > 6000:
            continue
        want, _ = oracle.block_hash(t.slice(a, b), mds)
        assert np.array_equal(pairs[offs[j]:offs[j + 1]], want)


def test_config5_full_size_learned_equals_plain():
    t, mds = synth.config5()
    with hb.Context(device=0) as ctx:
        ctx.load_table(0, t.n_rows, t.columns)
        for md in mds:
            ctx.add_md(md)
        ctx.plan("rule_data")
        pairs = ctx.block()
        ctx.plan("given")
        again = ctx.block()
    assert np.array_equal(pairs, again)
    idx = np.random.default_rng(4).choice(len(pairs), size=min(5000, len(pairs)), replace=False)
    assert oracle.check_pairs(t, mds, pairs[idx]).all()
