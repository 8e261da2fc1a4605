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


@pytest.mark.slow
def test_learned_tile_shape_skips_trial_runs_on_a_held_out_batch():
    """The committed tile-shape model (trained on the autotuner's logs of other
    batches) picks the batched form's tile shape without timing the eight
    candidates: on a held-out batch the first call is faster than with the
    autotuner, the chosen shape runs within 15 % of the autotuner's choice and
    the pairs are identical."""
    import os
    import statistics
    import time
    import torch
    model = np.load(os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                                 "paper_2410_04349_gb300", "tile_model.npy"))
    rng = np.random.default_rng(77)
    sizes = [int(x) for x in np.clip(np.round(np.exp(np.log(700) + 0.9 * rng.standard_normal(1200))), 20, 8000)]
    t, mds = synth.config4(n_jobs=len(sizes), sizes=sizes, seed=424242)
    res = {}
    for name, m in (("autotuned", None), ("learned", model)):
        with hb.Context(device=0) as ctx:
            ctx.load_table(0, t.n_rows, t.columns)
            for md in mds:
                ctx.add_md(md)
            if m is not None:
                ctx.set_tile_model(m)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            pairs, offs = ctx.block_batch(t.job_offsets)
            first = time.perf_counter() - t0
            shape = ctx.batch_tile()
            steady = []
            for _ in range(7):
                t0 = time.perf_counter()
                ctx.block_batch(t.job_offsets)
                steady.append(time.perf_counter() - t0)
            res[name] = (first, statistics.median(steady), shape, pairs, offs)
    fa, sa, sha, pa, oa = res["autotuned"]
    fl, sl, shl, pl, ol = res["learned"]
    assert sha[2] == 0 and shl[2] == 1
    assert np.array_equal(pa, pl) and np.array_equal(oa, ol)
    assert fl < fa
    assert sl <= 1.15 * sa, (res["autotuned"][:3], res["learned"][:3])
