"""Batched jobs (one persistent launch, CUDA graph replay) against the oracle
per job and against one launch sequence per job."""
import numpy as np
import pytest

import oracle
import synth
from paper_2410_04349_gb300 import hb

pytestmark = pytest.mark.gpu


def _batch(t, mds, flags=0, tile=0, calls=1):
    with hb.Context(device=0, flags=flags, tile=tile) as ctx:
        ctx.load_table(0, t.n_rows, t.columns)
        for md in mds:
            ctx.add_md(md)
        outs = [ctx.block_batch(t.job_offsets) for _ in range(calls)]
        st = ctx.stats()
    return outs, st


def _jobs(n_jobs=40, seed=7):
    sizes = [int(x) for x in np.random.default_rng(seed).integers(1, 900, n_jobs)]
    sizes[3] = 1
    sizes[5] = 2
    return synth.config4(n_jobs=n_jobs, sizes=sizes)


def test_batch_matches_oracle_per_job_and_graph_replays():
    t, mds = _jobs()
    outs, st = _batch(t, mds, calls=3)
    pairs, offs = outs[0]
    cand_total = 0
    for j in range(len(t.job_offsets) - 1):
        a, b = t.job_offsets[j], t.job_offsets[j + 1]
        want, cand = oracle.block_hash(t.slice(a, b), mds)
        assert np.array_equal(pairs[offs[j]:offs[j + 1]], want), j
        cand_total += cand
    assert st["candidate_pairs"] == cand_total
    for p2, o2 in outs[1:]:           # replays of the captured graph
        assert np.array_equal(p2, pairs) and np.array_equal(o2, offs)


def test_batch_equals_per_job_launches():
    t, mds = _jobs(25, seed=9)
    (a,), _ = _batch(t, mds)
    (b,), _ = _batch(t, mds, flags=hb.FLAG_PER_JOB_LAUNCHES)
    (c,), _ = _batch(t, mds, flags=hb.FLAG_NO_GRAPH, tile=64)
    for x in (b, c):
        assert np.array_equal(a[0], x[0]) and np.array_equal(a[1], x[1])


def test_batch_rejects_bad_job_rows():
    t, mds = _jobs(8)
    with hb.Context(device=0) as ctx:
        ctx.load_table(0, t.n_rows, t.columns)
        for md in mds:
            ctx.add_md(md)
        bad = t.job_offsets.copy()
        bad[-1] += 1
        with pytest.raises(hb.HBError):
            ctx.block_batch(bad)
