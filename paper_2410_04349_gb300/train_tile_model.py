"""Train the batched form's tile-shape model and write tile_model.npy.

The batch autotuner logs, for each job-size signature it meets, the time of
every candidate tile shape.  This script runs hb_block_batch once (fresh
context, so the autotuner measures) on seeded synthetic batches of the
10,000-job workload's schema whose job counts, typical sizes and size spreads
vary, with the workload's rules and seeded random rule sets, gathers the
logged (features, log ms) rows and trains the tile-shape network on the GPU
(hb_train_tile_model).  The 10,000-job workload itself is not among them.

  python -m paper_2410_04349_gb300.train_tile_model [--out PATH]
"""
from __future__ import annotations

import argparse
import json
import math
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))

from paper_2410_04349_gb300 import hb  # noqa: E402


def job_sizes(n_jobs, typical, spread, seed, lo=20, hi=8000):
    rng = np.random.default_rng(seed)
    s = np.exp(math.log(typical) + spread * rng.standard_normal(n_jobs))
    return [int(x) for x in np.clip(np.round(s), lo, hi)]


def batches():
    """(sizes, rule set) of the training batches."""
    import synth
    out = []
    k = 0
    for n_jobs in (150, 600, 1500):
        for typical in (120, 500, 1500):
            for spread in (0.5, 1.2):
                sizes = job_sizes(n_jobs, typical, spread, seed=9000 + k)
                if sum(sizes) > 2_500_000:
                    continue
                rules = synth.c2_mds() if k % 2 == 0 else synth.random_rule_set(5000 + k, 4, [2, 3, 4], [0, 1], [5, 6])
                out.append((sizes, rules, 8000 + k))
                k += 1
    return out


def training_rows():
    import synth
    Xs, ys = [], []
    for sizes, rules, seed in batches():
        t, _ = synth.config4(n_jobs=len(sizes), sizes=sizes, seed=seed)
        with hb.Context(device=0) as ctx:
            ctx.load_table(0, t.n_rows, t.columns)
            for md in rules:
                ctx.add_md(md)
            ctx.block_batch(t.job_offsets)
            X, y = ctx.tile_log()
        Xs.append(X)
        ys.append(y)
    return np.concatenate(Xs), np.concatenate(ys)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=os.path.join(HERE, "tile_model.npy"))
    ap.add_argument("--epochs", type=int, default=2000)
    args = ap.parse_args()
    t0 = time.time()
    X, y = training_rows()
    with hb.Context(device=0) as ctx:
        loss = ctx.train_tile_model(X, y, epochs=args.epochs)
        params = ctx.get_tile_model()
    np.save(args.out, params.astype(np.float32))
    print(json.dumps({"rows": int(len(y)), "loss": float(loss), "seconds": round(time.time() - t0, 1),
                      "out": args.out}))


if __name__ == "__main__":
    main()
