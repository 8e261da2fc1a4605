"""Pins of the plan-replay work counter (algorithmic units per candidate pair
under a given plan): hand-computed counts on tiny tables, early exit at a
checkpoint, and agreement of the replayed verdict with the disjunction for
every predicate order."""
import itertools

import numpy as np
import pytest

import oracle
import synth
from synth import absdiff, ed, eq, jac


def _t(rows):
    return synth.table_from_rows(["k", "s", "x"], ["int32", "string", "fp32"], rows)


def test_units_by_hand_edit_distance():
    # one MD: k equal and ED(s) <= 2; the pair (0, 1) is the only candidate
    t = _t([(1, "abcdefgh", 0.0), (1, "abcdefghij", 0.0), (2, "zz", 0.0)])
    u = oracle.plan_units(t, [[eq(0), ed(1, 2)]], [ed(1, 2)])
    # |10 - 8| <= 2: filter 3 + ceil(8/64) * 10 * 16 = 160
    assert u == {"eq": 1, "owner": 1, "absdiff": 0, "ed": 163, "jaccard": 0, "candidates": 1, "total": 165}
    u = oracle.plan_units(t, [[eq(0), ed(1, 1)]], [ed(1, 1)])
    assert u["ed"] == 3   # |10 - 8| > 1: only the length filter


def test_units_by_hand_jaccard_and_multiword_edit_distance():
    long_a = "a" * 70 + "b"
    long_b = "a" * 70 + "c"
    t = _t([(1, long_a, 0.0), (1, long_b, 0.0)])
    u = oracle.plan_units(t, [[eq(0), ed(1, 3)]], [ed(1, 3)])
    assert u["ed"] == 3 + 2 * 71 * 16   # two 64-bit words of the shorter string
    # 3-grams: "aaa", "aab" vs "aaa", "aac": |A| = |B| = 2, size filter passes
    u = oracle.plan_units(t, [[eq(0), jac(1, 1, 2)]], [jac(1, 1, 2)])
    assert u["jaccard"] == 3 + (2 + 2) * 4


def test_checkpoint_stops_the_replay():
    # MD 0 is a witness at the pair (same x); MD 1's predicate is never evaluated
    t = _t([(1, "hello", 1.0), (1, "help", 1.0)])
    mds = [[eq(0), absdiff(2, 0.5)], [eq(0), ed(1, 2)]]
    u = oracle.plan_units(t, mds, [absdiff(2, 0.5), ed(1, 2)])
    assert u["absdiff"] == 3 and u["ed"] == 0 and u["owner"] == 2 and u["eq"] == 1
    # the other order evaluates ED first (it passes) and stops at MD 1's checkpoint
    u = oracle.plan_units(t, mds, [ed(1, 2), absdiff(2, 0.5)])
    assert u["ed"] == 3 + 1 * 5 * 16 and u["absdiff"] == 0


@pytest.mark.parametrize("seed", [3, 4])
def test_every_order_replays_to_the_same_verdicts(seed):
    t = synth.random_small(seed=seed, n=120, null_rate=0.1)
    mds = [[eq(2), ed(0, 2), absdiff(4, 0.3)], [eq(3), jac(1, 1, 2), ed(0, 2)], [eq(2), eq(3), jac(1, 3, 5)]]
    dp = [p for p in oracle.distinct_predicates(mds) if p[0] not in ("eq", "eq_prefix")]
    totals = set()
    for order in itertools.permutations(dp):
        u = oracle.plan_units(t, mds, list(order))   # raises if a verdict differs
        assert u["candidates"] == oracle.block_hash(t, mds)[1]
        totals.add(u["total"])
    assert len(totals) > 1   # the order changes the work, never the result
