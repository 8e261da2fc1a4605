"""Execution-plan generator, restated from Section 4 — TEST INFRASTRUCTURE ONLY.

Plain Python, written step by step from the paper:

  * sp(p, D)  : "Effectiveness" (Section 4.2): hash the A-values into k
                buckets; sp = norm(sqrt(1/k * sum_i (b_i - |D|/k)^2)).
  * cost(p, D): "Estimated cost" (Section 4.2): norm(sum of per-pair costs).
  * norm(.)   : the paper only says it maps into (0, 1]; reading used here:
                divide by the maximum over all predicates, and clamp a zero to
                1e-6 (if every value is zero, all become 1e-6).
  * ordering  : "Ordering scheme": cost-effectiveness (1 - sp) / cost,
                descending; ties broken by the lower predicate id.
  * tree      : "Constructing an execution tree": insert every MD's
                predicates, sorted by cost-effectiveness, from the root,
                reusing a child whose edge carries the same predicate.
  * wp(phi)   : product of sp over the MD's predicates (in the MD's written
                order), independence assumption of Section 4.2.
  * score(e)  : "Edge score": max wp over the MDs whose root-to-leaf path
                contains e.
  * DFS       : "Evaluating an execution plan" (Section 4.1): children in
                decreasing score; ties go to the child created first (the lower
                MD id, since MDs are inserted in id order).
  * path      : "Tree traversal on GPUs" (Section 5.1): the DFS order written
                out as a list of predicates with a checkpoint (CP) at the end of
                every rule.

Parity of this module is pinned by the paper's worked examples (ordering
example of Section 4.2, tree-construction example, edge-score example, DFS
example of Section 4.1) in tests/test_oracle_plan.py.
"""
from __future__ import annotations

import math

EPS = 1e-6


def norm(values):
    """Map non-negative numbers into (0, 1] by dividing by their maximum."""
    mx = max(values) if values else 0.0
    if mx <= 0.0:
        return [EPS for _ in values]
    return [max(v / mx, EPS) for v in values]


def bucket_stddev(counts, n_total):
    """sqrt(1/k * sum_i (b_i - |D|/k)^2) over the k bucket counts."""
    k = len(counts)
    mean = n_total / k
    return math.sqrt(sum((b - mean) ** 2 for b in counts) / k)


def sp_from_buckets(bucket_counts_per_pred, n_total):
    """sp for every predicate from its LSH bucket counts, normalised together."""
    return norm([bucket_stddev(c, n_total) for c in bucket_counts_per_pred])


def cost_effectiveness(sp, cost):
    return [(1.0 - s) / c for s, c in zip(sp, cost)]


def order_predicates(sp, cost):
    """Predicate ids sorted by cost-effectiveness, descending (ties: lower id)."""
    ce = cost_effectiveness(sp, cost)
    return sorted(range(len(sp)), key=lambda p: (-ce[p], p))


class Node:
    __slots__ = ("pred", "children", "mds", "leaf_md", "first_md", "score")

    def __init__(self, pred=None, first_md=None):
        self.pred = pred          # predicate on the edge from the parent (None at the root)
        self.children = []        # in creation order
        self.mds = []             # MDs whose root-to-leaf path passes through this node's edge
        self.leaf_md = []         # MDs whose leaf is this node
        self.first_md = first_md  # MD that created this node
        self.score = 0.0


def build_tree(mds, sp, cost):
    """Execution tree over MDs given as lists of predicate ids."""
    ce = cost_effectiveness(sp, cost)
    root = Node()
    for m, preds in enumerate(mds):
        seq = sorted(dict.fromkeys(preds), key=lambda p: (-ce[p], p))
        node = root
        for p in seq:
            child = next((c for c in node.children if c.pred == p), None)
            if child is None:
                child = Node(p, m)
                node.children.append(child)
            child.mds.append(m)
            node = child
        node.leaf_md.append(m)
    return root


def witness_prob(mds, sp):
    out = []
    for preds in mds:
        w = 1.0
        for p in preds:
            w *= sp[p]
        out.append(w)
    return out


def assign_scores(root, wp):
    stack = [root]
    while stack:
        n = stack.pop()
        for c in n.children:
            c.score = max(wp[m] for m in c.mds)
            stack.append(c)
    return root


def dfs(root):
    """Yield ("pred", p) when an edge is taken and ("cp", m) at a leaf."""
    out = []

    def visit(node):
        for m in node.leaf_md:
            out.append(("cp", m))
        for c in sorted(node.children, key=lambda c: (-c.score, c.first_md)):
            out.append(("pred", c.pred))
            visit(c)

    visit(root)
    return out


def plan(mds, sp, cost):
    """Full plan: (predicate order, tree, wp, MD order, sequential path)."""
    order = order_predicates(sp, cost)
    tree = build_tree(mds, sp, cost)
    wp = witness_prob(mds, sp)
    assign_scores(tree, wp)
    path = dfs(tree)
    md_order = [x for k, x in path if k == "cp"]
    return {"order": order, "tree": tree, "wp": wp, "md_order": md_order, "path": path}


def flatten_program(path, mds, skip=()):
    """The sequential path with every predicate kept at its first occurrence
    only (later occurrences reuse the first result, Section 5.1 "Reusing
    computation"), dropping predicates in ``skip`` (those already decided
    elsewhere).  Returns the predicate sequence and, per MD, the index of the
    MD's last remaining predicate in that sequence: once that predicate has
    been evaluated every predicate of the MD has a result, so this is where its
    checkpoint (CP) takes effect (-1 when the MD has no remaining predicate)."""
    seq = []
    pos = {}
    for kind, x in path:
        if kind == "pred" and x not in pos and x not in skip:
            pos[x] = len(seq)
            seq.append(x)
    cp = [max([pos[p] for p in preds if p not in skip], default=-1) for preds in mds]
    return seq, cp
