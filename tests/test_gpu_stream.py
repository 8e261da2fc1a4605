"""R x S with S streamed from host memory in chunks, against the oracle and
against the resident R x S path."""
import numpy as np
import pytest

import oracle
import synth
from paper_2410_04349_gb300 import hb

pytestmark = pytest.mark.gpu


def _stream(r, s, mds, chunk_bytes):
    with hb.Context(device=0, chunk_bytes=chunk_bytes) as ctx:
        ctx.load_table(0, r.n_rows, r.columns)
        for md in mds:
            ctx.add_md(md)
        got = ctx.block_stream(s.n_rows, s.columns)
        again = ctx.block_stream(s.n_rows, s.columns)
        st = ctx.stats()
    return got, again, st


@pytest.mark.parametrize("chunk_bytes", [0, 40_000, 300_000])
def test_stream_matches_oracle(chunk_bytes):
    r, s, mds = synth.config3(n_r=3000, n_s=9000, cards=(15, 150, 1500))
    got, again, st = _stream(r, s, mds, chunk_bytes)
    want, cand = oracle.block_hash(r, mds, S=s)
    assert np.array_equal(got, want)
    assert np.array_equal(again, want)
    assert st["candidate_pairs"] == cand


def test_stream_with_missing_values():
    r = synth.random_small(seed=51, n=500, null_rate=0.15)
    s = synth.random_small(seed=52, n=1500, null_rate=0.15)
    from synth import absdiff, ed, eq, eq_prefix, jac
    mds = [[eq(2), ed(0, 2)], [eq(3), jac(1, 1, 2)], [eq_prefix(1, 2), absdiff(4, 0.3)]]
    got, _, _ = _stream(r, s, mds, 20_000)
    assert np.array_equal(got, oracle.block_literal(r, mds, S=s))


def test_stream_equals_resident_r_x_s():
    r, s, mds = synth.config3(n_r=4000, n_s=12000, cards=(20, 200, 2000))
    got, _, _ = _stream(r, s, mds, 100_000)
    with hb.Context(device=0) as ctx:
        ctx.load_table(0, r.n_rows, r.columns)
        ctx.load_table(1, s.n_rows, s.columns)
        for md in mds:
            ctx.add_md(md)
        res = ctx.block()
    assert np.array_equal(got, res)


@pytest.mark.parametrize("chunk_bytes", [0, 40_000])
def test_stream_from_page_locked_memory(chunk_bytes):
    """S in page-locked host memory is DMA'd per array instead of packed: same pairs."""
    r, s, mds = synth.config3(n_r=3000, n_s=9000, cards=(15, 150, 1500))
    locked = hb.pin_columns(s.columns)
    with hb.Context(device=0, chunk_bytes=chunk_bytes) as ctx:
        ctx.load_table(0, r.n_rows, r.columns)
        for md in mds:
            ctx.add_md(md)
        got = ctx.block_stream(s.n_rows, locked)
        pageable = ctx.block_stream(s.n_rows, s.columns)
        again = ctx.block_stream(s.n_rows, locked)
    want, _ = oracle.block_hash(r, mds, S=s)
    assert np.array_equal(got, want)
    assert np.array_equal(pageable, want)
    assert np.array_equal(again, want)


def test_load_table_from_page_locked_memory():
    """hb_load_table of page-locked host columns (one DMA per array) equals the staged upload."""
    r = synth.random_small(seed=61, n=1500, null_rate=0.1)
    from synth import absdiff, ed, eq, jac
    mds = [[eq(2), ed(0, 2)], [eq(3), jac(1, 1, 2)], [eq(2), absdiff(4, 0.3)]]
    res = []
    for cols in (r.columns, hb.pin_columns(r.columns)):
        with hb.Context(device=0, chunk_bytes=16_384) as ctx:
            ctx.load_table(0, r.n_rows, cols)
            for md in mds:
                ctx.add_md(md)
            res.append(ctx.block())
    assert np.array_equal(res[0], res[1])
    assert np.array_equal(res[0], oracle.block_literal(r, mds))
