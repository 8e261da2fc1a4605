"""Digests that pin whole results at the benchmark's full sizes: the sha256 of
a generated relation (so a test can tell a different input from a different
result) and of a sorted pair list, plus the fixed row subset of the
10M-tuple configuration whose pairs are compared exactly."""
import hashlib
import json
import os

import numpy as np

GOLDEN_DIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def table_sha256(t) -> str:
    h = hashlib.sha256()
    for c in t.columns:
        h.update(c.type.encode())
        h.update(np.ascontiguousarray(c.data).tobytes())
        if c.offsets is not None:
            h.update(np.ascontiguousarray(c.offsets, np.uint32).tobytes())
        if c.valid is not None:
            h.update(np.ascontiguousarray(c.valid, np.uint8).tobytes())
    return h.hexdigest()


def pairs_sha256(pairs, job_offsets=None) -> str:
    """sha256 of the pairs packed as little-endian uint64 (tid1 << 32 | tid2),
    in the given order (sorted ascending for a whole result), followed by the
    job offsets (int64) of a batched result."""
    p = np.asarray(pairs, np.int64).reshape(-1, 2)
    packed = (p[:, 0].astype(np.uint64) << np.uint64(32)) | p[:, 1].astype(np.uint64)
    h = hashlib.sha256(packed.astype("<u8").tobytes())
    if job_offsets is not None:
        h.update(np.asarray(job_offsets, "<i8").tobytes())
    return h.hexdigest()


def c5_subset(n_rows: int, frac_num: int = 3, frac_den: int = 10) -> np.ndarray:
    """Rows i of the 10M-tuple table with (i * 2654435761 mod 2^32) below
    frac_num/frac_den of 2^32 (Knuth's multiplicative hash: a fixed, spread
    out 30 % of the rows).  Whether a pair is a candidate depends on its two
    tuples only, so the full run's pairs inside this subset must equal the
    pairs of the subset blocked on its own."""
    i = np.arange(n_rows, dtype=np.uint64)
    h = (i * np.uint64(2654435761)) & np.uint64(0xFFFFFFFF)
    return np.nonzero(h < np.uint64((frac_num << 32) // frac_den))[0].astype(np.int64)


def load(config: str):
    path = os.path.join(GOLDEN_DIR, f"fullsize_{config}.json")
    if not os.path.exists(path):
        return None
    return json.load(open(path))
