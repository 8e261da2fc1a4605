"""GPU parity of the general predicate forms of Section 2 against the oracle:
constants on either tuple, equality across two columns of one relation,
q-gram containment (asymmetric: the library evaluates the transpose of every
asymmetric MD in a self-join) and word-token Jaccard, on small tables with
missing values, on R x S, on a 20,000-tuple table of the benchmark's shape and
in the batched form."""
import numpy as np
import pytest

import oracle
import synth
from gpu_helpers import run_gpu
from paper_2410_04349_gb300 import hb
from synth import absdiff, const_eq, contain, ed, eq, jac, tjac
from test_oracle_general import _words_table

pytestmark = pytest.mark.gpu

RULES = [[eq(2, 3), tjac(0, 1, 2)],                        # t.k = s.h (two columns), token Jaccard
         [const_eq(4, "red"), eq(3), contain(1, 2, 3, q=2)],
         [eq(2), const_eq(3, 1, side=1), ed(0, 1)],
         [tjac(1, 2, 3), eq(4)]]


@pytest.mark.parametrize("seed", [11, 12, 13])
def test_general_rules_self_join(seed):
    t = _words_table(seed, n=160)
    got, st, info = run_gpu(t, RULES)
    want = oracle.block_literal(t, RULES)
    assert np.array_equal(got, want)
    assert info.n_mds > len(RULES)   # transposed copies of the asymmetric MDs


def test_general_rules_every_plan_mode():
    t = _words_table(14, n=120)
    want = oracle.block_literal(t, RULES)
    for mode in ("rule_data", "given", "random", "cost_first", "sel_first"):
        got, _, _ = run_gpu(t, RULES, mode=mode)
        assert np.array_equal(got, want), mode


def test_general_rules_r_x_s():
    r, s = _words_table(21, n=90), _words_table(22, n=110)
    mds = [[eq(2, 3), tjac(0, 1, 2)], [const_eq(4, "blue", side=1), eq(3), contain(0, 1, 2, q=2, side=1)],
           [const_eq(2, 2), tjac(1, 1, 1)]]
    got, _, _ = run_gpu(r, mds, S=s)
    assert np.array_equal(got, oracle.block_literal(r, mds, S=s))


def test_general_rules_benchmark_shape():
    # 20,000 tuples of the single-table schema: s1, s2 (words), k1, k2, k3 (Zipf keys), x1, x2, id
    t, _ = synth.config2(n=20000, cards=(20, 200, 2000))
    mds = [[eq(2), tjac(0, 1, 2)],                          # word tokens of s1
           [eq(2, 4), eq(3), ed(1, 3)],                     # t.k1 = s.k3: two int32 columns
           [const_eq(3, bytes(t.columns[3].value(0))), eq(2), contain(1, 4, 5)],
           [eq(3), eq(4), jac(0, 4, 5), absdiff(5, 0.5)]]
    got, st, _ = run_gpu(t, mds)
    want, cand = oracle.block_owned(t, mds)
    assert np.array_equal(got, want)
    assert st["candidate_pairs"] == cand
    assert len(want) > 0


def test_general_rules_batched():
    jobs = [_words_table(30 + j, n=n) for j, n in enumerate([40, 1, 2, 75, 130])]
    t = synth.concat(jobs)
    with hb.Context(device=0) as ctx:
        ctx.load_table(0, t.n_rows, t.columns)
        for md in RULES:
            ctx.add_md(md)
        pairs, offs = ctx.block_batch(t.job_offsets)
    for j, sub in enumerate(jobs):
        assert np.array_equal(pairs[offs[j]:offs[j + 1]], oracle.block_literal(sub, RULES)), j


def test_streamed_s_rejects_constants_and_tokens():
    r, s = _words_table(41, n=30), _words_table(42, n=30)
    with hb.Context(device=0) as ctx:
        ctx.load_table(0, r.n_rows, r.columns)
        ctx.add_md([const_eq(4, "red", side=1), eq(3)])
        with pytest.raises(hb.HBError) as e:
            ctx.block_stream(s.n_rows, s.columns)
        assert e.value.status == hb.HB_ERR_ARG


def test_invalid_general_predicates():
    t = _words_table(43, n=20)
    with hb.Context(device=0) as ctx:
        ctx.load_table(0, t.n_rows, t.columns)
        for bad in (("const_eq", 2, 2, 0, 0, 0, 0, 0.0, 2, 1),          # side must be 0 or 1
                    ("contain", 0, 0, 0, 5, 1, 2, 0.0, 0),              # q in 1..4
                    ("tjaccard", 0, 0, 0, 0, 3, 2, 0.0)):               # num <= den
            with pytest.raises(hb.HBError):
                ctx.add_md([bad])
        ctx.add_md([ed(0, 2, cs=1)])                                    # two columns in a similarity
        with pytest.raises(hb.HBError):
            ctx.plan("rule_data")
