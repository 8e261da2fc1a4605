"""Writes tests/golden/fullsize_<config>.json: the oracle's exact result at the
benchmark's full sizes, as the number of pairs, the sha256 of the sorted pair
list and the number of candidate pairs (pairs agreeing on every equality
predicate of some MD, each once).  Only the oracle and the seeded input
generator run here; nothing of the GPU library is imported.

  python tests/golden/make_fullsize.py c2 c3 c4 c5

c2: 1,000,000 tuples, 4 MDs (self-join).   c3: R 500,000 x S 2,000,000, 6 MDs.
c4: 10,000 independent jobs, each blocked alone (job-local row ids, pairs of
    job j after those of job j - 1).
c5: 10,000,000 tuples, 16 MDs: the candidate count of the whole table, and
    the pairs of a fixed 30 % row subset blocked on its own (see c5_subset).
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)
sys.path.insert(0, os.path.dirname(HERE))

import numpy as np  # noqa: E402

import oracle  # noqa: E402
import synth  # noqa: E402
from fullsize_digest import c5_subset, pairs_sha256, table_sha256  # noqa: E402


def write(config, d):
    d["config"] = config
    d["command"] = f"python tests/golden/make_fullsize.py {config}"
    d["oracle"] = "oracle.block_owned (owner-rule pass of the grouped oracle, host threads)"
    with open(os.path.join(HERE, f"fullsize_{config}.json"), "w") as f:
        json.dump(d, f, indent=1)
        f.write("\n")
    print(config, json.dumps(d), flush=True)


def c2():
    t, mds = synth.config2()
    t0 = time.time()
    pairs, cand = oracle.block_owned(t, mds)
    write("c2", {"input_sha256": table_sha256(t), "n_pairs": int(len(pairs)), "pairs_sha256": pairs_sha256(pairs),
                 "candidates": cand, "seconds": round(time.time() - t0, 1)})


def c3():
    r, s, mds = synth.config3()
    t0 = time.time()
    pairs, cand = oracle.block_owned(r, mds, S=s)
    write("c3", {"input_sha256": table_sha256(r) + ":" + table_sha256(s), "n_pairs": int(len(pairs)),
                 "pairs_sha256": pairs_sha256(pairs), "candidates": cand, "seconds": round(time.time() - t0, 1)})


def c4():
    t, mds = synth.config4()
    t0 = time.time()
    jo = t.job_offsets
    parts, offs, cand = [], [0], 0
    for j in range(len(jo) - 1):
        p, c = oracle.block_owned(t.slice(int(jo[j]), int(jo[j + 1])), mds)
        parts.append(p)
        offs.append(offs[-1] + len(p))
        cand += c
    pairs = np.concatenate(parts) if parts else np.zeros((0, 2), np.int64)
    write("c4", {"input_sha256": table_sha256(t), "n_jobs": len(jo) - 1, "n_pairs": int(len(pairs)),
                 "pairs_sha256": pairs_sha256(pairs, offs), "candidates": cand,
                 "seconds": round(time.time() - t0, 1)})


def c5():
    t, mds = synth.config5()
    t0 = time.time()
    _, cand = oracle.block_owned(t, mds, evaluate=False)
    rows = c5_subset(t.n_rows)
    pairs, cand_sub = oracle.block_owned(t.take(rows), mds)
    write("c5", {"input_sha256": table_sha256(t), "candidates": cand, "subset_rows": int(len(rows)),
                 "subset_rule": "i * 2654435761 mod 2^32 < 3/10 * 2^32", "subset_candidates": cand_sub,
                 "n_pairs": int(len(pairs)), "pairs_sha256": pairs_sha256(pairs),
                 "seconds": round(time.time() - t0, 1)})


if __name__ == "__main__":
    for name in sys.argv[1:] or ["c2", "c3", "c4", "c5"]:
        {"c2": c2, "c3": c3, "c4": c4, "c5": c5}[name]()
