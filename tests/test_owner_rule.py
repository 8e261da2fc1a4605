"""The owner rule that lets every candidate pair be evaluated once: an MD builds
blocks only if no lower-numbered MD's equality keys are a subset of its keys
("active"), and a pair is handled only in the block of the lowest-numbered MD
whose keys it matches.  Property test on random rule sets and key tables: each
pair that agrees on some MD's equality keys is owned exactly once, by an active
MD's block, and no other pair is owned."""
import itertools
import random


def _active(eqsets):
    return [m for m, s in enumerate(eqsets) if not any(eqsets[j] <= s for j in range(m))]


def _matched_keys(a, b):
    return frozenset(k for k, (x, y) in enumerate(zip(a, b)) if x is not None and x == y)


def test_each_candidate_pair_has_exactly_one_owner():
    rng = random.Random(7)
    for trial in range(300):
        n_keys = rng.randint(1, 5)
        n_md = rng.randint(1, 6)
        eqsets = [frozenset(rng.sample(range(n_keys), rng.randint(0, n_keys))) for _ in range(n_md)]
        n = rng.randint(2, 25)
        card = rng.randint(1, 4)
        rows = [[None if rng.random() < 0.1 else rng.randrange(card) for _ in range(n_keys)] for _ in range(n)]
        active = _active(eqsets)
        for i, j in itertools.combinations(range(n), 2):
            E = _matched_keys(rows[i], rows[j])
            alive = [m for m in range(n_md) if eqsets[m] <= E]
            # blocks of active MD a that hold the pair, and those among them that own it
            holders = [a for a in active if eqsets[a] <= E]
            owners = [a for a in holders if a == min(alive)]
            if alive:
                assert len(owners) == 1, (trial, eqsets, E)
                assert min(alive) in active
            else:
                assert not holders and not owners


def test_dominated_rules_never_own():
    # a rule whose keys include a lower-numbered rule's keys adds no blocks
    eqsets = [frozenset({0, 1}), frozenset({1}), frozenset({0, 1, 2}), frozenset({2})]
    assert _active(eqsets) == [0, 1, 3]
