"""Pins of the oracle's single predicates against definitions that do not go
through the oracle's own code: edit distance by breadth-first search over edit
operations, q-gram Jaccard by Python sets and exact fractions, |a-b| <= delta
by numpy binary32 arithmetic."""
import itertools
import random
from fractions import Fraction

import numpy as np
import pytest

import oracle


def bfs_edit_distance(a: str, b: str, alphabet: str) -> int:
    """Fewest single-character insertions, deletions and substitutions turning
    a into b (the definition of the Levenshtein distance), by BFS."""
    if a == b:
        return 0
    maxlen = max(len(a), len(b)) + 1
    seen = {a}
    frontier = [a]
    d = 0
    while frontier:
        d += 1
        nxt = []
        for s in frontier:
            cands = set()
            for i in range(len(s) + 1):
                for c in alphabet:
                    cands.add(s[:i] + c + s[i:])
            for i in range(len(s)):
                cands.add(s[:i] + s[i + 1:])
                for c in alphabet:
                    cands.add(s[:i] + c + s[i + 1:])
            for t in cands:
                if len(t) > maxlen or t in seen:
                    continue
                if t == b:
                    return d
                seen.add(t)
                nxt.append(t)
        frontier = nxt
    raise AssertionError("unreachable")


def test_edit_distance_matches_bfs_definition_exhaustive():
    alphabet = "ab"
    words = [""] + ["".join(p) for n in range(1, 5) for p in itertools.product(alphabet, repeat=n)]
    for a in words:
        for b in words:
            assert oracle.edit_distance(a, b) == bfs_edit_distance(a, b, alphabet), (a, b)


def test_edit_distance_three_letter_alphabet_sample():
    rng = random.Random(7)
    for _ in range(200):
        a = "".join(rng.choice("abc") for _ in range(rng.randint(0, 4)))
        b = "".join(rng.choice("abc") for _ in range(rng.randint(0, 4)))
        assert oracle.edit_distance(a, b) == bfs_edit_distance(a, b, "abc"), (a, b)


def test_edit_distance_known_values_and_properties():
    assert oracle.edit_distance("kitten", "sitting") == 3
    assert oracle.edit_distance("", "abc") == 3
    assert oracle.edit_distance("flaw", "lawn") == 2
    rng = random.Random(3)
    for _ in range(300):
        a = bytes(rng.randrange(256) for _ in range(rng.randint(0, 80)))
        b = bytes(rng.randrange(256) for _ in range(rng.randint(0, 80)))
        c = bytes(rng.randrange(256) for _ in range(rng.randint(0, 20)))
        dab = oracle.edit_distance(a, b)
        assert dab == oracle.edit_distance(b, a)
        assert abs(len(a) - len(b)) <= dab <= max(len(a), len(b))
        assert oracle.edit_distance(a, a) == 0
        assert oracle.edit_distance(a, c) <= dab + oracle.edit_distance(b, c)
        # appending the same byte string to both never changes more than it costs
        assert oracle.edit_distance(a + c, b + c) <= dab


def py_jaccard(a: bytes, b: bytes, q: int):
    A = {a[i:i + q] for i in range(len(a) - q + 1)}
    B = {b[i:i + q] for i in range(len(b) - q + 1)}
    return len(A), len(B), len(A & B)


def test_qgram_sets_hand_computed():
    # "abcabc" -> {abc, bca, cab}; "abcd" -> {abc, bcd}; common {abc}
    assert oracle.qgram_sets("abcabc", "abcd") == (3, 2, 1)
    assert oracle.qgram_sets("ab", "abc") == (0, 1, 0)
    assert oracle.qgram_sets("", "") == (0, 0, 0)
    assert oracle.qgram_sets("aaaa", "aaa") == (1, 1, 1)


def test_jaccard_integer_boundaries():
    # abcdef: abc bcd cde def (4); abcdefg adds efg (5): J = 4/5 exactly
    assert oracle.jaccard_ge("abcdef", "abcdefg", 4, 5)
    assert not oracle.jaccard_ge("abcdef", "abcdefg", 81, 100)
    assert oracle.jaccard_ge("abcabc", "abcd", 1, 4)        # J = 1/4
    assert not oracle.jaccard_ge("abcabc", "abcd", 26, 100)
    # both sets empty: 0 * den >= num * 0 holds; one empty: fails for num > 0
    assert oracle.jaccard_ge("ab", "cd", 4, 5)
    assert not oracle.jaccard_ge("ab", "abc", 4, 5)
    assert oracle.jaccard_ge("ab", "abc", 0, 5)


def test_jaccard_against_python_sets_random():
    rng = random.Random(11)
    for _ in range(500):
        a = bytes(rng.choice(b"abcd ") for _ in range(rng.randint(0, 30)))
        b = bytes(rng.choice(b"abcd ") for _ in range(rng.randint(0, 30)))
        q = rng.choice([1, 2, 3, 4])
        na, nb, ni = py_jaccard(a, b, q)
        assert oracle.qgram_sets(a, b, q) == (na, nb, ni)
        num, den = rng.choice([(4, 5), (7, 10), (1, 2), (1, 1), (0, 1)])
        u = na + nb - ni
        expect = (Fraction(ni, u) >= Fraction(num, den)) if u else True
        assert oracle.jaccard_ge(a, b, num, den, q) == expect


def test_absdiff_binary32_boundaries():
    f = np.float32
    assert oracle.absdiff_le(1.0, 1.5, 0.5)
    assert not oracle.absdiff_le(1.0, float(np.nextafter(f(1.5), f(2))), 0.5)
    assert oracle.absdiff_le(-0.0, 0.0, 0.0)
    assert not oracle.absdiff_le(float("nan"), 1.0, 1e30)
    assert not oracle.absdiff_le(1.0, float("inf"), 1e30)
    # 1e8 has binary32 spacing 8: the difference is 8 exactly
    assert not oracle.absdiff_le(1e8, 1e8 + 8, 7.99)
    assert oracle.absdiff_le(1e8, 1e8 + 8, 8.0)
    rng = np.random.default_rng(5)
    a = rng.lognormal(3, 1, 4000).astype(np.float32)
    b = (a + rng.normal(0, 0.5, 4000)).astype(np.float32)
    d = rng.choice(np.array([0.25, 0.5, 1.0], np.float32), 4000)
    expect = np.abs(a - b) <= d          # numpy binary32 subtract, round to nearest even
    got = [oracle.absdiff_le(float(x), float(y), float(z)) for x, y, z in zip(a, b, d)]
    assert (np.array(got) == expect).all()
