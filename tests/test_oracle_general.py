"""Pins of the general predicate forms of Section 2 ("Predicates": t.A = c,
t.A = s.B, any symmetric or asymmetric similarity measure) in the oracle:
constants on either tuple, equality across two columns of one relation,
q-gram containment (asymmetric) and word-token Jaccard, each against a plain
Python definition with exact fractions; and the self-join reading for
asymmetric rules (a pair {i, j} is reported when some MD is a witness at
(t_i, t_j) or at (t_j, t_i)), including the identity that the second
valuation of an MD equals the first valuation of its transpose."""
from fractions import Fraction
import itertools
import random

import numpy as np
import pytest

import oracle
import synth
from synth import absdiff, const_eq, contain, ed, eq, jac, tjac


def py_tokens(s: bytes):
    return {t for t in s.split(b" ") if t}


def py_grams(s: bytes, q: int):
    return {s[i:i + q] for i in range(len(s) - q + 1)}


def py_pred(t, p, i, j, S=None):
    S = S or t
    kind, ct, cs, k, q, num, den, delta = p[:8]
    side = p[8] if len(p) > 8 else 0
    if kind == "const_eq":
        col, row = (t.columns[ct], i) if side == 0 else (S.columns[cs], j)
        v = col.value(row)
        want = p[9].encode() if isinstance(p[9], str) else p[9]
        return v is not None and v == want
    a, b = t.columns[ct].value(i), S.columns[cs].value(j)
    if a is None or b is None:
        return False
    if kind == "eq":
        return a == b
    if kind == "ed":
        return oracle.edit_distance(a, b) <= k
    if kind == "jaccard":
        A, B = py_grams(a, q), py_grams(b, q)
        return len(A | B) == 0 or Fraction(len(A & B), len(A | B)) >= Fraction(num, den)
    if kind == "absdiff":
        return oracle.absdiff_le(a, b, delta)
    if kind == "contain":
        A, B = py_grams(a, q), py_grams(b, q)
        D, E = (A, B) if side == 0 else (B, A)
        return len(D & E) * den >= num * len(D)
    if kind == "tjaccard":
        A, B = py_tokens(a), py_tokens(b)
        return len(A & B) * den >= num * len(A | B)
    raise ValueError(kind)


def py_witness(t, mds, i, j, S=None):
    return any(all(py_pred(t, p, i, j, S) for p in md) for md in mds)


def py_block(t, mds, S=None):
    out = []
    if S is not None:
        for i in range(t.n_rows):
            for j in range(S.n_rows):
                if py_witness(t, mds, i, j, S):
                    out.append((i, j))
    else:
        for i in range(t.n_rows):
            for j in range(i + 1, t.n_rows):
                if py_witness(t, mds, i, j) or py_witness(t, mds, j, i):
                    out.append((i, j))
    return np.array(out, np.int64).reshape(-1, 2)


def transpose(md):
    """The MD with the roles of its two tuple variables exchanged."""
    out = []
    for p in md:
        p = list(p)
        p[1], p[2] = p[2], p[1]
        if p[0] in ("const_eq", "contain"):
            p[8] = 1 - p[8]
        out.append(tuple(p))
    return out


def _words_table(seed, n=70, null_rate=0.1):
    rng = random.Random(seed)
    words = [b"ab", b"cd", b"abc", b"x", b"cdab", b"", b"ab cd"]
    rows = []
    for _ in range(n):
        def s():
            if rng.random() < null_rate:
                return None
            k = rng.randint(0, 4)
            return b" ".join(rng.choice(words) for _ in range(k)) + (b" " if rng.random() < 0.2 else b"")
        rows.append((s(), s(), rng.choice([None, 1, 2, 3]) if null_rate else rng.choice([1, 2, 3]),
                     rng.choice([None, 1, 2, 3]) if null_rate else rng.choice([1, 2, 3]),
                     rng.choice(["red", "blue", None])))
    return synth.table_from_rows(["a", "b", "k", "h", "c"], ["string", "string", "int32", "int32", "string"], rows)


def test_token_jaccard_against_python_sets():
    rng = random.Random(5)
    alphabet = [b"a", b"b", b" ", b"ab"]
    for _ in range(400):
        a = b"".join(rng.choice(alphabet) for _ in range(rng.randint(0, 8)))
        b = b"".join(rng.choice(alphabet) for _ in range(rng.randint(0, 8)))
        t = synth.table_from_rows(["s"], ["string"], [(a,), (b,)])
        for num, den in ((1, 2), (2, 3), (1, 1), (0, 1)):
            got = oracle.pred_verdicts(t, tjac(0, num, den), [(0, 1)])[0]
            A, B = py_tokens(a), py_tokens(b)
            want = len(A & B) * den >= num * len(A | B)
            assert got == want, (a, b, num, den)
    # hand cases: runs of spaces separate, empty and all-space strings have no tokens
    t = synth.table_from_rows(["s"], ["string"], [(b"ab  cd ",), (b"cd ab",), (b"   ",), (b"",)])
    assert oracle.pred_verdicts(t, tjac(0, 1, 1), [(0, 1)])[0] == 1
    assert oracle.pred_verdicts(t, tjac(0, 1, 1), [(2, 3)])[0] == 1   # empty vs empty: 0 >= 0
    assert oracle.pred_verdicts(t, tjac(0, 1, 2), [(0, 2)])[0] == 0


def test_containment_is_asymmetric():
    # G3("abcd") = {abc, bcd} is inside G3("abcde"), not the other way round
    t = synth.table_from_rows(["s"], ["string"], [(b"abcd",), (b"abcde",)])
    assert oracle.pred_verdicts(t, contain(0, 1, 1), [(0, 1)])[0] == 1
    assert oracle.pred_verdicts(t, contain(0, 1, 1), [(1, 0)])[0] == 0
    assert oracle.pred_verdicts(t, contain(0, 1, 1, side=1), [(1, 0)])[0] == 1
    assert oracle.pred_verdicts(t, contain(0, 2, 3), [(1, 0)])[0] == 1     # 2 of 3 grams
    assert oracle.pred_verdicts(t, contain(0, 3, 4), [(1, 0)])[0] == 0
    rng = random.Random(8)
    for _ in range(300):
        a = bytes(rng.choice(b"ab") for _ in range(rng.randint(0, 7)))
        b = bytes(rng.choice(b"ab") for _ in range(rng.randint(0, 7)))
        t = synth.table_from_rows(["s"], ["string"], [(a,), (b,)])
        for side in (0, 1):
            for num, den in ((1, 2), (3, 4), (1, 1)):
                p = contain(0, num, den, q=2, side=side)
                assert oracle.pred_verdicts(t, p, [(0, 1)])[0] == py_pred(t, p, 0, 1)


def test_constants_on_either_tuple():
    t = _words_table(3)
    for i, j in itertools.product(range(12), repeat=2):
        for p in (const_eq(2, 2), const_eq(2, 3, side=1), const_eq(4, "red"), const_eq(4, "blue", side=1)):
            assert oracle.pred_verdicts(t, p, [(i, j)])[0] == py_pred(t, p, i, j)


@pytest.mark.parametrize("seed", [11, 12])
def test_general_rules_match_python_loop(seed):
    t = _words_table(seed)
    mds = [[eq(2, 3), tjac(0, 1, 2)],                       # t.k = s.h (two columns), token Jaccard
           [const_eq(4, "red"), eq(3), contain(1, 2, 3, q=2)],
           [eq(2), const_eq(3, 1, side=1), ed(0, 1)],
           [tjac(1, 2, 3), eq(4)]]
    want = py_block(t, mds)
    assert np.array_equal(oracle.block_literal(t, mds), want)
    assert np.array_equal(oracle.block_hash(t, mds)[0], want)
    assert np.array_equal(oracle.block_owned(t, mds, threads=3)[0], want)
    # the second valuation of an asymmetric MD is the first valuation of its transpose
    both = mds + [transpose(md) for md in mds]
    first_only = set()
    for i in range(t.n_rows):
        for j in range(i + 1, t.n_rows):
            if py_witness(t, both, i, j):
                first_only.add((i, j))
    assert first_only == set(map(tuple, want.tolist()))


def test_general_rules_r_x_s():
    r, s = _words_table(21, n=30), _words_table(22, n=35)
    mds = [[eq(2, 3), tjac(0, 1, 2)], [const_eq(4, "blue", side=1), eq(3), contain(0, 1, 2, q=2, side=1)]]
    want = py_block(r, mds, S=s)
    assert np.array_equal(oracle.block_literal(r, mds, S=s), want)
    assert np.array_equal(oracle.block_hash(r, mds, S=s)[0], want)
    assert np.array_equal(oracle.block_owned(r, mds, S=s)[0], want)


def test_symmetric_rules_keep_one_valuation():
    # with symmetric predicates only, the self-join result is that of the first valuation
    t = synth.random_small(seed=3, n=80, null_rate=0.1)
    mds = [[eq(2), ed(0, 2)], [eq(3), jac(1, 1, 2), absdiff(4, 0.3)]]
    lit = oracle.block_literal(t, mds)
    one = [(i, j) for i in range(t.n_rows) for j in range(i + 1, t.n_rows) if py_witness(t, mds, i, j)]
    assert lit.tolist() == [list(x) for x in one]
