"""Train the blocker's cost model on its own logs and write cost_model.npy.

Section 4.2 ("Shallow NNs", "Estimated cost") trains a shallow network offline
on historical logs of predicate evaluations.  This script produces those logs
by running the library's instrumented evaluation (every predicate of every
rule on every candidate pair, hb_log_predicates with profile = 1) over
seeded synthetic workloads shaped like the single-table (1M tuples), R x S
(500K x 2M) and batched (jobs of 3,000-20,000 tuples) benchmarks, each with its
own rules and seeded random rule sets, then fits both networks on the GPU with
the library's forward, backward and Adam kernels (hb_train_cost_model) and
saves the weights (2 x HB_MLP_PARAMS float32) next to this file.

  python -m paper_2410_04349_gb300.train_cost_model [--out PATH] [--epochs N]

The 10M-tuple, 16-rule workload that the learned plan is compared on is not
among the training data.
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))

from paper_2410_04349_gb300 import hb, learn  # noqa: E402


def training_rows():
    """(X [n, 32], log_cost [n], logit_pass [n]) from logs of the training workloads."""
    import synth
    Xs, ycs, yss = [], [], []

    def rows(table, sets, S=None):
        with hb.Context(device=0) as ctx:
            ctx.load_table(0, table.n_rows, table.columns)
            if S is not None:
                ctx.load_table(1, S.n_rows, S.columns)
            for mds in sets:
                ctx.clear_mds()
                for md in mds:
                    ctx.add_md(md)
                ctx.plan("rule_data")
                X, yc, ys = learn.collect(ctx)
                Xs.append(X)
                ycs.append(yc)
                yss.append(ys)

    t2, m2 = synth.config2()
    rows(t2, [m2] + [synth.random_rule_set(100 + i, 4, [2, 3, 4], [0, 1], [5, 6]) for i in range(16)])
    r3, s3, m3 = synth.config3()
    rows(r3, [m3] + [synth.random_rule_set(200 + i, 4, [2, 3, 4], [0, 1], [5, 6]) for i in range(8)], S=s3)
    sizes = [20000, 16000, 12000, 9000, 7000, 5000, 4000, 3000]
    t4, m4 = synth.config4(n_jobs=len(sizes), sizes=sizes)
    for j in range(len(sizes)):
        sub = t4.slice(t4.job_offsets[j], t4.job_offsets[j + 1])
        rows(sub, [m4] + [synth.random_rule_set(300 + 10 * j + i, 4, [2, 3, 4], [0, 1], [5, 6], n_keys=(1, 2))
                          for i in range(3)])
    return np.concatenate(Xs), np.concatenate(ycs), np.concatenate(yss)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=os.path.join(HERE, "cost_model.npy"))
    ap.add_argument("--epochs", type=int, default=1500)
    args = ap.parse_args()
    t0 = time.time()
    X, yc, ys = training_rows()
    with hb.Context(device=0) as ctx:
        loss = learn.train(ctx, X, yc, ys, epochs=args.epochs)
        params = ctx.get_cost_model()
    np.save(args.out, params.astype(np.float32))
    print(json.dumps({"rows": int(len(X)), "loss_cost": float(loss[0]), "loss_sel": float(loss[1]),
                      "seconds": round(time.time() - t0, 1), "out": args.out}))


if __name__ == "__main__":
    main()
