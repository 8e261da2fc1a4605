"""Root-edge hash partitioning of Section 5.3 ("Data partitioning") — TEST
INFRASTRUCTURE ONLY (imported by ``tests/`` alone).

The paper hashes every tuple with s functions, one per child of the root of
the execution tree, each built from the predicate on that root edge, and
compares only tuples that one function puts in the same partition (a tuple
carries the branch of the function that placed it).  Readings taken here:

  * the equality predicates of an MD are its block keys and sit at the top of
    its path, so the root edge of an MD is its first equality predicate in the
    written order (same-column in a self-join; either relation's column in
    R x S); an MD without one hangs from a similarity root, for which the
    paper's remark lets a partition pull every other one: that branch puts
    all tuples in one partition;
  * the branches are the distinct root predicates in order of first
    appearance over the MDs;
  * the hash of a value is 32-bit FNV-1a (Fowler, Noll, Vo; offset basis
    2166136261, prime 16777619) of its bytes — a string's bytes (its first k
    for a prefix equality), an int32's four little-endian bytes — taken
    modulo the number of partitions m; a missing value is in no partition;
  * a pair is a candidate when some branch puts both tuples in one partition;
    every MD holds its root predicate, so every pair some MD accepts is a
    candidate, and the blocking result is the plain one of Section 2.

``candidates`` counts the candidate pairs by brute force over all pairs.
"""
from __future__ import annotations

import numpy as np

FNV_OFFSET = 2166136261
FNV_PRIME = 16777619


def fnv1a32(data: bytes) -> int:
    """32-bit FNV-1a of a byte string: for each byte, xor it in, then multiply
    by the FNV prime modulo 2^32."""
    h = FNV_OFFSET
    for b in data:
        h ^= b
        h = (h * FNV_PRIME) & 0xFFFFFFFF
    return h


def root_keys(mds, self_join=True):
    """Per MD, its root equality key (kind, col_t, col_s, prefix) or None."""
    out = []
    for md in mds:
        key = None
        for p in md:
            kind, ct, cs, k = p[0], p[1], p[2], p[3]
            if kind not in ("eq", "eq_prefix"):
                continue
            if self_join and ct != cs:   # two columns of one relation: not a block key
                continue
            key = (kind, ct, cs, k if kind == "eq_prefix" else -1)
            break
        out.append(key)
    return out


def branches(mds, self_join=True):
    """Distinct root keys in order of first appearance (None: the branch that
    puts all tuples in one partition)."""
    out = []
    for k in root_keys(mds, self_join):
        if k not in out:
            out.append(k)
    return out


def value_bytes(col, i, prefix=-1):
    """The bytes a row's value hashes with (None when the value is missing)."""
    v = col.value(i)
    if v is None:
        return None
    if col.type == "string":
        return v if prefix < 0 else v[:prefix]
    if col.type == "int32":
        return int(v).to_bytes(4, "little", signed=True)
    raise ValueError("equality keys are string or int32 columns")


def partition_ids(table, key, m, side):
    """Partition of every row of one relation under one branch: an int64 array
    with -1 for rows in no partition; the all-tuples branch gives 0 for all."""
    n = table.n_rows
    if key is None:
        return np.zeros(n, dtype=np.int64)
    _, ct, cs, prefix = key
    col = table.columns[ct if side == 0 else cs]
    out = np.empty(n, dtype=np.int64)
    for i in range(n):
        b = value_bytes(col, i, prefix)
        out[i] = -1 if b is None else fnv1a32(b) % m
    return out


def candidates(R, mds, m, S=None):
    """Pairs that some branch puts in one partition: (t_i, t_j) with i < j for
    a self-join, every (t_i, s_j) for R x S.  Brute force over all pairs."""
    self_join = S is None
    other = R if self_join else S
    nr, ns = R.n_rows, other.n_rows
    co = np.zeros((nr, ns), dtype=bool)
    for key in branches(mds, self_join):
        a = partition_ids(R, key, m, 0)
        b = partition_ids(other, key, m, 1)
        co |= (a[:, None] == b[None, :]) & (a[:, None] >= 0)
    if self_join:
        co = np.triu(co, k=1)
    return int(co.sum())
