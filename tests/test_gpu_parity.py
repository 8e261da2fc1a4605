"""GPU pair sets against the CPU oracle, element by element (tolerance 0)."""
import json
import os

import numpy as np
import pytest

import oracle
import synth
from synth import absdiff, ed, eq, eq_prefix, jac

from gpu_helpers import committed_model, as_set, run_gpu

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("tile", [32, 64])
def test_config1_pairs_and_candidates(tile):
    t, mds = synth.config1()
    got, st, _ = run_gpu(t, mds, tile=tile)
    want, cand = oracle.block_hash(t, mds)
    assert np.array_equal(got, want)
    assert st["candidate_pairs"] == cand
    assert np.array_equal(oracle.block_literal(t, mds), want)


def small_mds():
    return [[eq(2), ed(0, 2)], [eq(3), jac(1, 1, 2)], [eq_prefix(1, 2), absdiff(4, 0.3)],
            [eq(2), eq(3), ed(1, 5)], [eq(3), jac(0, 2, 3, q=2), absdiff(4, 1.0)]]


@pytest.mark.parametrize("seed", [1, 2, 3, 4])
@pytest.mark.parametrize("null_rate", [0.0, 0.2])
def test_random_small_with_nulls(seed, null_rate):
    t = synth.random_small(seed=seed, n=700, null_rate=null_rate)
    mds = small_mds()
    got, st, _ = run_gpu(t, mds)
    want = oracle.block_literal(t, mds)
    assert np.array_equal(got, want)
    _, cand = oracle.block_hash(t, mds)
    assert st["candidate_pairs"] == cand


def test_paper_table1_fixture():
    d = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "table1_products.json")))
    t = synth.table_from_rows(d["columns"], d["types"], d["rows"])
    for k in (8, 9):
        mds = [[eq(5), eq(2), eq(3), ed(1, k)], [eq(3), jac(4, 1, 2)], [ed(6, k), jac(4, 1, 2)]]
        got, _, _ = run_gpu(t, mds)
        want = oracle.block_literal(t, mds)
        assert np.array_equal(got, want)
        assert ((0, 3) in as_set(got)) == (k >= 9)


@pytest.mark.parametrize("mode", ["rule_data", "given", "random", "cost_first", "sel_first", "learned"])
def test_every_plan_mode_gives_the_same_set(mode):
    t, mds = synth.config2(n=30000, cards=(30, 300, 3000))
    model = committed_model() if mode == "learned" else None
    got, _, info = run_gpu(t, mds, mode=mode, model=model)
    want, _ = oracle.block_hash(t, mds)
    assert np.array_equal(got, want)
    if mode == "learned":
        assert info.mode == 1   # the committed model was applied, not the rule-data fallback


def test_r_x_s_small():
    r = synth.random_small(seed=41, n=400, null_rate=0.1)
    s = synth.random_small(seed=42, n=650, null_rate=0.1)
    mds = small_mds()
    got, st, _ = run_gpu(r, mds, S=s)
    want = oracle.block_literal(r, mds, S=s)
    assert np.array_equal(got, want)
    _, cand = oracle.block_hash(r, mds, S=s)
    assert st["candidate_pairs"] == cand


def test_r_x_s_config3_shape():
    r, s, mds = synth.config3(n_r=6000, n_s=15000, cards=(20, 200, 2000))
    got, st, _ = run_gpu(r, mds, S=s)
    want, cand = oracle.block_hash(r, mds, S=s)
    assert np.array_equal(got, want)
    assert st["candidate_pairs"] == cand


def test_config2_shape_many_tiles():
    t, mds = synth.config2(n=40000, cards=(40, 400, 4000))
    got, st, _ = run_gpu(t, mds)
    want, cand = oracle.block_hash(t, mds)
    assert np.array_equal(got, want)
    assert st["candidate_pairs"] == cand
    assert st["tiles"] > 1000


def test_empty_and_single_row():
    t = synth.random_small(seed=3, n=0)
    got, st, _ = run_gpu(t, small_mds())
    assert got.shape == (0, 2) and st["candidate_pairs"] == 0
    t = synth.random_small(seed=3, n=1)
    got, st, _ = run_gpu(t, small_mds())
    assert got.shape == (0, 2)


def test_one_huge_block_grows_the_output_slab():
    # 2500 identical rows: every pair is a witness (3.1M pairs > initial slab)
    rows = [("abcdef", "x y z", 1, "k", 1.0)] * 2500
    t = synth.table_from_rows(["a", "b", "k", "c", "x"], ["string", "string", "int32", "string", "fp32"], rows)
    mds = [[eq(2), ed(0, 1)]]
    got, st, _ = run_gpu(t, mds, out_capacity=1000)
    n = 2500
    assert len(got) == n * (n - 1) // 2
    assert st["candidate_pairs"] == n * (n - 1) // 2
    assert np.array_equal(got[:3], np.array([[0, 1], [0, 2], [0, 3]]))


def test_rule_without_equality_compares_all_pairs():
    t = synth.random_small(seed=8, n=500, alphabet_small=True)
    mds = [[ed(0, 2)], [jac(1, 3, 5), absdiff(4, 0.2)]]
    got, st, _ = run_gpu(t, mds)
    assert np.array_equal(got, oracle.block_literal(t, mds))
    assert st["candidate_pairs"] == 500 * 499 // 2


@pytest.mark.parametrize("k", [0, 1, 3, 4, 6, 12, 31])
def test_edit_distance_thresholds(k):
    t = synth.random_small(seed=100 + k, n=600, alphabet_small=True)
    mds = [[eq(2), ed(0, k)], [eq(3), ed(1, k)]]
    got, _, _ = run_gpu(t, mds)
    assert np.array_equal(got, oracle.block_literal(t, mds))


@pytest.mark.parametrize("q", [1, 2, 3, 4])
def test_jaccard_gram_lengths(q):
    t = synth.random_small(seed=200 + q, n=600)
    mds = [[eq(2), jac(1, 1, 3, q=q)], [eq(3), jac(0, 3, 5, q=q)], [eq(2), jac(1, 0, 1, q=q)]]
    got, _, _ = run_gpu(t, mds)
    assert np.array_equal(got, oracle.block_literal(t, mds))


def test_long_strings_and_empty_strings():
    rng = np.random.default_rng(5)
    rows = []
    base = "".join(rng.choice(list("abcdefgh"), 900))
    for i in range(160):
        kind = i % 4
        if kind == 0:
            s = base                      # > 64 grams: the block-sort path
        elif kind == 1:
            s = base[: 300 + i] + "q"
        elif kind == 2:
            s = ""                        # empty string: no grams
        else:
            s = "".join(rng.choice(list("ab"), 3))
        rows.append((s, s[:40], i % 3, "c", float(i % 5)))
    t = synth.table_from_rows(["a", "b", "k", "c", "x"], ["string", "string", "int32", "string", "fp32"], rows)
    mds = [[eq(2), jac(0, 4, 5)], [eq(3), ed(1, 2)], [eq(2), jac(0, 1, 1, q=2)]]
    got, _, _ = run_gpu(t, mds)
    assert np.array_equal(got, oracle.block_literal(t, mds))


def test_results_are_deterministic():
    t, mds = synth.config2(n=20000, cards=(20, 200, 2000))
    a, _, _ = run_gpu(t, mds)
    b, _, _ = run_gpu(t, mds)
    c, _, _ = run_gpu(t, mds, tile=64)
    assert np.array_equal(a, b) and np.array_equal(a, c)


def _edited(rng, s, n_edits, alphabet):
    s = list(s)
    for _ in range(n_edits):
        op = rng.integers(3)
        p = int(rng.integers(len(s) + 1))
        if op == 0 and p < len(s):
            s[p] = rng.choice(alphabet)
        elif op == 1:
            s.insert(p, rng.choice(alphabet))
        elif p < len(s):
            del s[p]
    return "".join(s)


@pytest.mark.parametrize("k", [2, 5, 12, 31])
def test_edit_distance_across_pattern_words(k):
    """Near-duplicates of strings whose shorter side spans one 64-byte word, two
    words, or more (the banded fallback), edited around the threshold."""
    rng = np.random.default_rng(17)
    alphabet = list("abcd")
    rows = []
    group = 0
    for length in (30, 63, 64, 65, 100, 127, 128, 129, 200, 300):
        for rep in range(2):
            base = "".join(rng.choice(alphabet, length))
            for v in range(7):
                rows.append((_edited(rng, base, int(rng.integers(0, 2 * k + 6)), alphabet), group))
            group += 1
    t = synth.table_from_rows(["s", "g"], ["string", "int32"], rows)
    mds = [[eq(1), ed(0, k)]]
    got, _, _ = run_gpu(t, mds)
    want = oracle.block_literal(t, mds)
    assert 0 < len(want) < 20 * 21   # some in-group pairs pass, not all
    assert np.array_equal(got, want)


@pytest.mark.parametrize("q", [2, 3, 4])
def test_jaccard_across_gram_list_sizes(q):
    """Gram lists sorted by one thread (<= 64 grams), one warp (65..256) and one
    block (more), with near-duplicates around the threshold."""
    rng = np.random.default_rng(23 + q)
    alphabet = list("abcdefgh")
    rows = []
    group = 0
    for length in (30, 66, 67, 120, 200, 258, 259, 300):
        for rep in range(2):
            base = "".join(rng.choice(alphabet, length))
            for v in range(6):
                rows.append((_edited(rng, base, int(rng.integers(0, length // 6 + 2)), alphabet), group))
            group += 1
    t = synth.table_from_rows(["s", "g"], ["string", "int32"], rows)
    mds = [[eq(1), jac(0, 3, 4, q=q)]]
    got, _, _ = run_gpu(t, mds)
    want = oracle.block_literal(t, mds)
    assert 0 < len(want) < 16 * 15
    assert np.array_equal(got, want)
