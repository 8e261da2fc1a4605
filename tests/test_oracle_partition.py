"""Pins of the root-edge hash partitioning oracle (Section 5.3, "Data
partitioning"): the FNV-1a hash against the published test vectors of its
authors, the candidate count against closed forms (one partition; the branch
of all tuples), against exact grouping when no two values collide, against a
pair-by-pair restatement for R x S, and completeness (every pair some MD
accepts is a candidate)."""
import itertools

import pytest

import oracle
import oracle.partition as op
import synth


def test_fnv1a32_published_vectors():
    assert op.fnv1a32(b"") == 0x811C9DC5
    assert op.fnv1a32(b"a") == 0xE40C292C
    assert op.fnv1a32(b"foobar") == 0xBF9CF968


def test_root_edges_follow_the_written_order():
    s, k1, k2 = 0, 2, 3
    mds = [[synth.ed(s, 1), synth.eq(k2), synth.eq(k1)],
           [synth.eq(k1), synth.jac(s, 1, 2)],
           [synth.ed(s, 2)],
           [synth.eq(0, 1), synth.eq(k1)],        # two columns of one relation: not a block key
           [synth.eq_prefix(s, 3), synth.eq(k2)]]
    keys = op.root_keys(mds)
    assert keys == [("eq", k2, k2, -1), ("eq", k1, k1, -1), None, ("eq", k1, k1, -1), ("eq_prefix", s, s, 3)]
    assert op.branches(mds) == [("eq", k2, k2, -1), ("eq", k1, k1, -1), None, ("eq_prefix", s, s, 3)]
    # in R x S a cross-column equality is a block key
    assert op.root_keys([[synth.eq(0, 1)]], self_join=False) == [("eq", 0, 1, -1)]


def _keyed_table(vals):
    rows = [(v, f"s{i}") for i, v in enumerate(vals)]
    return synth.table_from_rows(["k", "s"], ["int32", "string"], rows)


def test_one_partition_holds_every_present_value():
    vals = [3, None, 7, 7, None, 1, 9, 2, None, 5, 5, 5]
    t = _keyed_table(vals)
    present = sum(v is not None for v in vals)
    assert op.candidates(t, [[synth.eq(0), synth.ed(1, 1)]], m=1) == present * (present - 1) // 2
    # an MD without an equality predicate adds the branch of all tuples
    mds = [[synth.eq(0), synth.ed(1, 1)], [synth.ed(1, 2)]]
    assert op.candidates(t, mds, m=5) == len(vals) * (len(vals) - 1) // 2


def test_without_collisions_partitions_are_the_equality_groups():
    t = synth.random_small(3, n=250, null_rate=0.1)
    k, c = 2, 3   # int key over 7 values, string key over 20
    m = 2_147_483_647
    for key_col in (k, c):
        col = t.columns[key_col]
        hashes = {}
        for i in range(t.n_rows):
            b = op.value_bytes(col, i)
            if b is not None:
                hashes.setdefault(op.fnv1a32(b) % m, set()).add(b)
        assert all(len(v) == 1 for v in hashes.values())   # no collision among these values
    mds = [[synth.eq(k), synth.ed(0, 2)], [synth.eq(c), synth.eq(k), synth.jac(1, 1, 2)]]
    # pairs sharing a present k, or a present c (each MD's root: k, then c)
    want = 0
    for i, j in itertools.combinations(range(t.n_rows), 2):
        share = False
        for key_col in (k, c):
            a, b = t.columns[key_col].value(i), t.columns[key_col].value(j)
            share |= a is not None and a == b
        want += share
    assert op.candidates(t, mds, m=m) == want


def test_cross_relation_count_pair_by_pair():
    R = synth.random_small(5, n=60, null_rate=0.15)
    S = synth.random_small(6, n=45, null_rate=0.15)
    mds = [[synth.eq_prefix(0, 2), synth.ed(0, 3)], [synth.eq(2), synth.jac(1, 1, 3)]]
    m = 4
    want = 0
    for i in range(R.n_rows):
        for j in range(S.n_rows):
            hit = False
            a, b = R.columns[0].value(i), S.columns[0].value(j)
            if a is not None and b is not None:
                hit |= op.fnv1a32(a[:2]) % m == op.fnv1a32(b[:2]) % m
            a, b = R.columns[2].value(i), S.columns[2].value(j)
            if a is not None and b is not None:
                hit |= op.fnv1a32(int(a).to_bytes(4, "little", signed=True)) % m == \
                    op.fnv1a32(int(b).to_bytes(4, "little", signed=True)) % m
            want += hit
    assert op.candidates(R, mds, m=m, S=S) == want


@pytest.mark.parametrize("seed", [11, 12, 13])
def test_every_accepted_pair_is_a_candidate(seed):
    t = synth.random_small(seed, n=300, null_rate=0.05)
    mds = [[synth.eq(2), synth.ed(0, 3)], [synth.eq(3), synth.jac(1, 1, 3)], [synth.eq_prefix(0, 1), synth.eq(2)]]
    pairs, _ = oracle.block_hash(t, mds)
    assert len(pairs) > 0
    for m in (1, 3, 17):
        ids = [op.partition_ids(t, key, m, 0) for key in op.branches(mds)]
        for i, j in pairs:
            assert any(p[i] >= 0 and p[i] == p[j] for p in ids)
    # one partition per function puts every present pair together
    assert op.candidates(t, mds, m=1) >= max(op.candidates(t, mds, m=m) for m in (3, 17))
