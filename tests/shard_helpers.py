"""The owner rank of a sharded evaluation, written from its specification in
include/hb.h (hb_set_shard), and the expected shard of every pair of a
self-join result.  Shared by the CPU (gloo) and GPU sharding tests."""
import numpy as np

M32 = 0xFFFFFFFF


def fmix32(h):
    """The 32-bit finaliser of MurmurHash3."""
    h &= M32
    h ^= h >> 16
    h = (h * 0x85EBCA6B) & M32
    h ^= h >> 13
    h = (h * 0xC2B2AE35) & M32
    h ^= h >> 16
    return h


def shard_of(md, row, world):
    return fmix32(row ^ ((md * 0x9E3779B9) & M32)) % world


def _key_values(table, md):
    """Per row, the tuple of the MD's equality-key values (None when some is
    missing); equality keys are the 'eq' and 'eq_prefix' predicates."""
    keys = [p for p in md if p[0] in ("eq", "eq_prefix")]
    out = []
    for i in range(table.n_rows):
        vals = []
        for p in keys:
            v = table.columns[p[1]].value(i)
            if v is None:
                vals = None
                break
            if p[0] == "eq_prefix":
                v = v[:p[3]]
            vals.append(v)
        out.append(None if vals is None else tuple(vals))
    return out


def expected_shards(table, mds, pairs, world):
    """Rank of every pair (i, j) of a self-join: the pair belongs to the lowest
    MD whose equality keys all agree on it; its group is the set of rows with
    those key values; the rank is shard_of(md, smallest row of the group)."""
    per_md = [_key_values(table, md) for md in mds]
    group_min = []
    for kv in per_md:
        first = {}
        for i, v in enumerate(kv):
            if v is not None and v not in first:
                first[v] = i
        group_min.append(first)
    ranks = np.empty(len(pairs), np.int64)
    for k, (i, j) in enumerate(np.asarray(pairs).tolist()):
        owner = None
        for m, kv in enumerate(per_md):
            if kv[i] is not None and kv[i] == kv[j]:
                owner = m
                break
        assert owner is not None, "a result pair agrees on no MD's equality keys"
        ranks[k] = shard_of(owner, group_min[owner][per_md[owner][i]], world)
    return ranks
