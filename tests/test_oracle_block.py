"""Pins of the oracle's blocking result: the paper's worked examples on its
Table 1, a pure-Python nested loop built from the (separately pinned) single
predicates, and invariants of the definition (symmetry, union over rules,
monotonicity in thresholds, grouped == naive)."""
import json
import os

import numpy as np
import pytest

import oracle
import synth
from synth import absdiff, ed, eq, eq_prefix, jac

GOLD = os.path.join(os.path.dirname(__file__), "golden", "table1_products.json")


def table1():
    d = json.load(open(GOLD))
    t = synth.table_from_rows(d["columns"], d["types"], d["rows"])
    return t, d


def paper_mds(k_ed=9, jd=(1, 2)):
    # columns: 0 pno, 1 pname, 2 price, 3 sname, 4 description, 5 color, 6 saddress
    phi1 = [eq(5), eq(2), eq(3), ed(1, k_ed)]
    phi2 = [eq(3), jac(4, *jd)]
    phi3 = [ed(6, k_ed), jac(4, *jd)]
    return [phi1, phi2, phi3]


def test_table1_example3_witnesses():
    t, d = table1()
    phi1 = paper_mds()[0:1]
    for i, j in d["facts"]["example3_phi1_witness"]:
        assert oracle.check_pairs(t, phi1, [(i, j)])[0] == 1
    for i, j in d["facts"]["example3_phi1_not_witness"]:
        assert oracle.check_pairs(t, phi1, [(i, j)])[0] == 0
        # t2.price is missing: the price predicate alone already fails
        assert oracle.pred_verdicts(t, eq(2), [(i, j)])[0] == 0


def test_table1_t1_t5_example():
    t, d = table1()
    for i, j in d["facts"]["example_t1_t5_sname_holds"]:
        assert oracle.pred_verdicts(t, eq(3), [(i, j)])[0] == 1
    for i, j in d["facts"]["example_t1_t5_description_jd_fails"]:
        for num, den in [(0, 1), (1, 10), (1, 2)]:
            assert oracle.pred_verdicts(t, jac(4, num, den), [(i, j)])[0] == 0


def test_table1_ed_threshold_reading():
    """phi1 is a witness at (t1, t4) in Example 3; byte Levenshtein between the
    two product names is 9, so the (unstated) threshold must admit 9."""
    t, _ = table1()
    assert oracle.check_pairs(t, paper_mds(9)[0:1], [(0, 3)])[0] == 1
    assert oracle.check_pairs(t, paper_mds(8)[0:1], [(0, 3)])[0] == 0
    full = oracle.block_literal(t, paper_mds(9))
    assert [0, 3] in full.tolist()
    assert [1, 2] not in oracle.block_literal(t, paper_mds(9)[0:1]).tolist()


def py_pred(t, p, i, j, S=None):
    S = S or t
    kind, ct, cs, k, q, num, den, delta = p
    a, b = t.columns[ct].value(i), S.columns[cs].value(j)
    if a is None or b is None:
        return False
    if kind == "eq":
        return a == b
    if kind == "eq_prefix":
        return a[:k] == b[:k]
    if kind == "ed":
        return oracle.edit_distance(a, b) <= k
    if kind == "jaccard":
        return oracle.jaccard_ge(a, b, num, den, q)
    if kind == "absdiff":
        return oracle.absdiff_le(a, b, delta)
    raise ValueError(kind)


def py_block(t, mds, S=None):
    out = []
    nS = (S or t).n_rows
    for i in range(t.n_rows):
        for j in (range(nS) if S else range(i + 1, nS)):
            if any(all(py_pred(t, p, i, j, S) for p in md) for md in mds):
                out.append((i, j))
    return np.array(out, np.int64).reshape(-1, 2)


def py_candidates(t, mds, S=None):
    nS = (S or t).n_rows
    n = 0
    for i in range(t.n_rows):
        for j in (range(nS) if S else range(i + 1, nS)):
            if any(all(py_pred(t, p, i, j, S) for p in md if p[0] in ("eq", "eq_prefix")) for md in mds):
                n += 1
    return n


def small_mds():
    # columns of synth.random_small: 0 a, 1 b, 2 k, 3 c, 4 x
    return [[eq(2), ed(0, 2)], [eq(3), jac(1, 1, 2)], [eq_prefix(1, 2), absdiff(4, 0.3)], [eq(2), eq(3), ed(1, 5)]]


@pytest.mark.parametrize("null_rate", [0.0, 0.15])
def test_literal_and_hash_match_python_loop(null_rate):
    t = synth.random_small(seed=17, n=90, null_rate=null_rate)
    mds = small_mds()
    lit = oracle.block_literal(t, mds)
    py = py_block(t, mds)
    assert np.array_equal(lit, py)
    h, cand = oracle.block_hash(t, mds)
    assert np.array_equal(h, py)
    assert cand == py_candidates(t, mds)


def test_rs_matches_python_loop():
    r = synth.random_small(seed=21, n=40, null_rate=0.1)
    s = synth.random_small(seed=22, n=55, null_rate=0.1)
    mds = small_mds()
    lit = oracle.block_literal(r, mds, S=s)
    assert np.array_equal(lit, py_block(r, mds, S=s))
    h, cand = oracle.block_hash(r, mds, S=s)
    assert np.array_equal(h, lit)
    assert cand == py_candidates(r, mds, S=s)


def test_rule_without_equality_contributes_all_pairs():
    t = synth.random_small(seed=5, n=60)
    mds = [[ed(0, 3)], [eq(2), jac(1, 1, 2)]]
    lit = oracle.block_literal(t, mds)
    h, cand = oracle.block_hash(t, mds)
    assert np.array_equal(lit, h)
    assert cand == 60 * 59 // 2


def test_symmetry_and_self_join_relation():
    t = synth.random_small(seed=9, n=70, null_rate=0.1)
    mds = small_mds()
    ordered = oracle.block_literal(t, mds, S=t)
    s = set(map(tuple, ordered.tolist()))
    for i, j in s:
        assert (j, i) in s
    upper = sorted((i, j) for i, j in s if i < j)
    assert upper == [tuple(x) for x in oracle.block_literal(t, mds).tolist()]


def test_union_over_rules():
    t, mds = synth.config1()
    full = set(map(tuple, oracle.block_hash(t, mds)[0].tolist()))
    parts = set()
    for md in mds:
        parts |= set(map(tuple, oracle.block_hash(t, [md])[0].tolist()))
    assert full == parts


def test_threshold_monotonicity():
    t = synth.random_small(seed=31, n=120)
    prev = None
    for k in range(0, 6):
        cur = set(map(tuple, oracle.block_hash(t, [[eq(2), ed(0, k)]])[0].tolist()))
        if prev is not None:
            assert prev <= cur
        prev = cur
    prev = None
    for num in [9, 7, 5, 3, 1]:
        cur = set(map(tuple, oracle.block_hash(t, [[eq(3), jac(1, num, 10)]])[0].tolist()))
        if prev is not None:
            assert prev <= cur
        prev = cur
    prev = None
    for d in [0.0, 0.1, 0.5, 2.0]:
        cur = set(map(tuple, oracle.block_hash(t, [[eq(2), absdiff(4, d)]])[0].tolist()))
        if prev is not None:
            assert prev <= cur
        prev = cur


def test_config1_literal_equals_hash():
    t, mds = synth.config1()
    lit = oracle.block_literal(t, mds)
    h, cand = oracle.block_hash(t, mds)
    assert np.array_equal(lit, h)
    assert len(lit) > 0 and cand >= len(lit)


@pytest.mark.parametrize("null_rate", [0.0, 0.15])
def test_owner_pass_matches_python_loop(null_rate):
    """The owner-rule pass (each candidate looked at once, big groups split
    over threads, q-gram sets built once per row) gives the nested loop's
    pairs and the brute-force candidate count, self-join and R x S."""
    t = synth.random_small(seed=41, n=90, null_rate=null_rate)
    mds = small_mds()
    py = py_block(t, mds)
    for threads in (1, 3):
        got, cand = oracle.block_owned(t, mds, threads=threads)
        assert np.array_equal(got, py)
        assert cand == py_candidates(t, mds)
    assert oracle.block_owned(t, mds, evaluate=False)[1] == cand
    r = synth.random_small(seed=43, n=40, null_rate=null_rate)
    s = synth.random_small(seed=44, n=55, null_rate=null_rate)
    got, cand = oracle.block_owned(r, mds, S=s, threads=2)
    assert np.array_equal(got, py_block(r, mds, S=s))
    assert cand == py_candidates(r, mds, S=s)


def test_owner_pass_rule_without_equality_and_big_groups():
    # one key value for every row: one group of 2,200 rows is cut into many
    # work ranges; an MD without equality owns the pairs the others miss
    t = synth.random_small(seed=47, n=2200)
    t.columns[2].data[:] = 3
    mds = [[eq(2), eq(3), ed(0, 1)], [jac(1, 7, 10)], [eq(2), absdiff(4, 0.05)]]
    want, cand_h = oracle.block_hash(t, mds)
    got, cand = oracle.block_owned(t, mds, threads=4)
    assert np.array_equal(got, want)
    assert cand == cand_h == 2200 * 2199 // 2


def test_owner_pass_config1_equals_literal():
    t, mds = synth.config1()
    got, cand = oracle.block_owned(t, mds)
    assert np.array_equal(got, oracle.block_literal(t, mds))
    assert cand == oracle.block_hash(t, mds)[1]
