"""Host-side fault injection (no GPU fault): HB_FAIL_ALLOC_AFTER=N makes the
(N+1)-th device or page-locked allocation of a context fail once.  For every N
up to the number of allocations a call sequence makes, the failing call must
return HB_ERR_OOM, and repeating it in the same context must give the oracle's
pairs."""
import numpy as np
import pytest

import oracle
import synth
from paper_2410_04349_gb300 import hb

pytestmark = pytest.mark.gpu

MDS = [[synth.eq(2), synth.ed(0, 3)], [synth.eq(3), synth.jac(1, 1, 3)], [synth.eq_prefix(0, 2), synth.absdiff(4, 0.3)]]


def _sweep(monkeypatch, run, want, max_n=400):
    met = 0
    for n in range(max_n):
        monkeypatch.setenv("HB_FAIL_ALLOC_AFTER", str(n))
        hit = []

        def step(f):
            try:
                return f()
            except hb.HBError as e:
                assert e.status == hb.HB_ERR_OOM, e
                hit.append(n)
                return f()

        with hb.Context(device=0) as ctx:
            pairs = run(ctx, step)
        assert np.array_equal(pairs, want), n
        if not hit:
            return met   # n is past the last allocation of the sequence
        met += 1
    raise AssertionError("the sequence kept allocating")


def test_self_join(monkeypatch):
    t = synth.random_small(61, n=900, null_rate=0.05)
    want, _ = oracle.block_hash(t, MDS)

    def run(ctx, step):
        step(lambda: ctx.load_table(0, t.n_rows, t.columns))
        for md in MDS:
            ctx.add_md(md)
        step(lambda: ctx.plan("rule_data"))
        return step(ctx.block)

    assert _sweep(monkeypatch, run, want) >= 10


def test_cross_relation_and_stream(monkeypatch):
    R = synth.random_small(62, n=500, null_rate=0.05)
    S = synth.random_small(63, n=700, null_rate=0.05)
    want, _ = oracle.block_hash(R, MDS, S=S)

    def run_resident(ctx, step):
        step(lambda: ctx.load_table(0, R.n_rows, R.columns))
        step(lambda: ctx.load_table(1, S.n_rows, S.columns))
        for md in MDS:
            ctx.add_md(md)
        return step(ctx.block)

    def run_stream(ctx, step):
        step(lambda: ctx.load_table(0, R.n_rows, R.columns))
        for md in MDS:
            ctx.add_md(md)
        return step(lambda: ctx.block_stream(S.n_rows, S.columns))

    assert _sweep(monkeypatch, run_resident, want) >= 10
    assert _sweep(monkeypatch, run_stream, want) >= 10
