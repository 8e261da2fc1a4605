"""Status codes and messages of the C-ABI on invalid input (no GPU fault is
involved: every case is rejected on the host)."""
import numpy as np
import pytest

import synth
from paper_2410_04349_gb300 import hb
from synth import absdiff, ed, eq, jac

pytestmark = pytest.mark.gpu


def _ctx_with(t):
    ctx = hb.Context(device=0)
    ctx.load_table(0, t.n_rows, t.columns)
    return ctx


def test_calls_out_of_order():
    with hb.Context(device=0) as ctx:
        with pytest.raises(hb.HBError) as e:
            ctx.block()
        assert e.value.status == hb.HB_ERR_STATE
        t, mds = synth.config1(n=50)
        ctx.load_table(0, t.n_rows, t.columns)
        with pytest.raises(hb.HBError) as e:
            ctx.plan()
        assert e.value.status == hb.HB_ERR_STATE


@pytest.mark.parametrize("bad", [
    [ed(0, 32)], [ed(0, -1)], [jac(0, 1, 2, q=5)], [jac(0, 3, 2)], [absdiff(3, -1.0)],
    [("eq_prefix", 0, 0, 0, 0, 0, 0, 0.0)], [ed(0, 33)],
])
def test_invalid_predicates_rejected(bad):
    t, _ = synth.config1(n=50)
    with _ctx_with(t) as ctx:
        with pytest.raises(hb.HBError) as e:
            ctx.add_md(bad)
        assert e.value.status == hb.HB_ERR_ARG


@pytest.mark.parametrize("md,why", [
    ([eq(3)], "equality on fp32"),
    ([ed(1, 2)], "edit distance on int32"),
    ([eq(9)], "missing column"),
    ([("ed", 0, 2, 2, 0, 0, 0, 0.0)], "self-join across columns"),
])
def test_rules_that_do_not_fit_the_schema(md, why):
    t, _ = synth.config1(n=50)
    with _ctx_with(t) as ctx:
        ctx.add_md(md)
        with pytest.raises(hb.HBError) as e:
            ctx.plan()
        assert e.value.status == hb.HB_ERR_ARG, why


def test_too_many_rules_and_predicates():
    t, _ = synth.config1(n=50)
    with _ctx_with(t) as ctx:
        for m in range(64):
            ctx.add_md([eq(1), ed(0, m % 31)])
        with pytest.raises(hb.HBError):
            ctx.add_md([eq(1)])
        with pytest.raises(hb.HBError):
            ctx.add_md([eq(1)] * 11)


def test_bad_tables_rejected():
    with hb.Context(device=0) as ctx:
        c = synth.Column("s", "string", np.frombuffer(b"abcdef", np.uint8).copy(), np.array([0, 4, 2, 6], np.uint32))
        with pytest.raises(hb.HBError) as e:
            ctx.load_table(0, 3, [c])
        assert e.value.status == hb.HB_ERR_ARG and "decrease" in str(e.value)
        with pytest.raises(hb.HBError):
            ctx.load_table(0, 1 << 30, [])
        with pytest.raises(hb.HBError):
            ctx.load_table(2, 0, [])


def test_jaccard_string_too_long_is_an_error():
    s = "ab" * 5000                      # 9999 grams > 8192
    t = synth.table_from_rows(["a", "k"], ["string", "int32"], [(s, 1), (s, 1), ("xy", 2)])
    with _ctx_with(t) as ctx:
        ctx.add_md([eq(1), jac(0, 1, 2)])
        with pytest.raises(hb.HBError) as e:
            ctx.block()
        assert e.value.status == hb.HB_ERR_ARG and "8192" in str(e.value)
