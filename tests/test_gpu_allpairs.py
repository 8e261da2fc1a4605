"""The all-pairs path at scale (Section 5.2's setting: an MD without an equality
predicate compares every pair): 200,000 tuples of the benchmark's schema, one
rule |x1 - x1'| <= 0.02 and ED(s1) <= 3 (2.0e10 candidate pairs, evaluated by
the tile queue in one all-tuple block), next to a blocked rule.  The candidate
count is exact by construction (every pair); the pairs are compared with the
oracle on a fixed 5 % row subset (whether a pair is a candidate depends on its
two tuples only)."""
import numpy as np
import pytest

import oracle
import synth
from fullsize_digest import c5_subset
from gpu_helpers import run_gpu
from synth import absdiff, ed, eq, jac

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


def test_all_pairs_rule_on_200k_tuples():
    n = 200_000
    t, _ = synth.config2(n=n)
    mds = [[absdiff(5, 0.02), ed(0, 3)], [eq(3), eq(4), jac(1, 7, 10)]]
    got, st, _ = run_gpu(t, mds)
    assert st["candidate_pairs"] == n * (n - 1) // 2
    rows = c5_subset(n, 1, 20)
    pos = np.full(n, -1, np.int64)
    pos[rows] = np.arange(len(rows))
    a, b = pos[got[:, 0]], pos[got[:, 1]]
    keep = (a >= 0) & (b >= 0)
    sub = np.stack([a[keep], b[keep]], axis=1)
    sub = sub[np.lexsort((sub[:, 1], sub[:, 0]))]
    want, cand = oracle.block_owned(t.take(rows), mds)
    assert cand == len(rows) * (len(rows) - 1) // 2
    assert np.array_equal(sub, want)
    assert len(want) > 0
