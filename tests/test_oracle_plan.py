"""Pins of the plan oracle by the worked examples of Sections 4.1-4.2.

Predicates of Example 2 (ids): 0 color=, 1 price=, 2 sname=, 3 pname~ED,
4 description~JD, 5 saddress~ED.  phi1 = {0,1,2,3}, phi2 = {2,4}, phi3 = {5,4}.
"""
import math
import random

import oracle.plan as P

MDS = [[0, 1, 2, 3], [2, 4], [5, 4]]
# sp values of the examples: sp(color) = 1 (all tuples are Gray), sp(pname) =
# 0.4, sp(sname) = 0.4, sp(description) = 0.2; sp(price) = 0.3 so that
# wp(phi1) = 1 * 0.3 * 0.4 * 0.4 = 0.048 as the edge-score example assumes.
SP = [1.0, 0.3, 0.4, 0.4, 0.2, 0.3]
# cost(color) = 0.1 and cost(pname) = 0.6 as in the ordering example; the rest
# make sname the first predicate of phi1, as the tree-construction example has it.
COST = [0.1, 0.2, 0.1, 0.6, 0.9, 0.5]


def test_ordering_example_pname_before_color():
    ce = P.cost_effectiveness(SP, COST)
    assert ce[0] == 0.0                        # (1 - 1) / 0.1
    assert ce[3] > ce[0]
    order = P.order_predicates(SP, COST)
    assert order.index(3) < order.index(0)


def test_tree_construction_example_shares_sname_node():
    tree = P.build_tree(MDS[:2], SP, COST)
    assert [c.pred for c in tree.children] == [2]         # N1: p_sname
    n1 = tree.children[0]
    assert n1.mds == [0, 1]
    # phi1's path continues below N1; phi2 adds N5 = p_description under N1
    assert [c.pred for c in n1.children] == [1, 4]
    n5 = n1.children[1]
    assert n5.leaf_md == [1] and n5.children == []
    # phi1's path has length |X| = 4 and every predicate once
    path, node = [], n1
    path.append(node.pred)
    node = node.children[0]
    while True:
        path.append(node.pred)
        if node.leaf_md:
            break
        node = node.children[0]
    assert sorted(path) == [0, 1, 2, 3] and node.leaf_md == [0]


def test_edge_score_example():
    wp = P.witness_prob(MDS, SP)
    assert math.isclose(wp[1], 0.08)            # 0.4 * 0.2
    assert math.isclose(wp[0], 0.048)
    tree = P.assign_scores(P.build_tree(MDS, SP, COST), wp)
    n1 = next(c for c in tree.children if c.pred == 2)
    assert math.isclose(n1.score, 0.08)         # max(0.048, 0.08)


def test_dfs_example_checks_phi2_phi1_phi3():
    r = P.plan(MDS, SP, COST)
    assert r["md_order"] == [1, 0, 2]
    # the root has two children and sname (higher score) is explored first
    assert len(r["tree"].children) == 2
    assert r["path"][0] == ("pred", 2)


def test_flattened_path_reuses_shared_predicates():
    r = P.plan(MDS, SP, COST)
    seq, cp = P.flatten_program(r["path"], MDS)
    assert sorted(seq) == sorted(set(seq)) == [0, 1, 2, 3, 4, 5]
    assert seq.index(4) < seq.index(5)          # description first met under N1, reused by phi3
    for m, preds in enumerate(MDS):
        assert cp[m] == max(seq.index(p) for p in preds)
    seq2, cp2 = P.flatten_program(r["path"], MDS, skip={0, 1, 2})
    assert set(seq2) == {3, 4, 5} and cp2[1] == seq2.index(4)


def test_sp_formula_extremes():
    n, k = 1000, 10
    all_in_one = [n] + [0] * (k - 1)
    even = [n // k] * k
    assert P.bucket_stddev(even, n) == 0.0
    assert math.isclose(P.bucket_stddev(all_in_one, n), math.sqrt(((n - n / k) ** 2 + (k - 1) * (n / k) ** 2) / k))
    sp = P.sp_from_buckets([all_in_one, even], n)
    assert sp[0] == 1.0 and sp[1] == P.EPS


def test_plan_is_a_permutation_for_random_rules():
    rng = random.Random(2)
    for _ in range(50):
        n_p = rng.randint(1, 12)
        mds = [rng.sample(range(n_p), rng.randint(1, min(5, n_p))) for _ in range(rng.randint(1, 8))]
        sp = [rng.random() for _ in range(n_p)]
        cost = [rng.uniform(0.01, 1) for _ in range(n_p)]
        r = P.plan(mds, sp, cost)
        assert sorted(r["md_order"]) == list(range(len(mds)))
        seq, cp = P.flatten_program(r["path"], mds)
        assert sorted(seq) == sorted(set(p for md in mds for p in md))
