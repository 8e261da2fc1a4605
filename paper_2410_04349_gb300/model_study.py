"""The model study of Section 6 (Exp-3, "Shallow model N") for the paper's
per-pair cost model N (hb_train_pair_model, layer sizes 8-2-6-1): on a sample
of tuple pairs per predicate, logged by the library's per-pair timing kernel,

  (1) noise: N is trained with beta % of the training labels replaced by
      values drawn uniformly between the smallest and largest training label,
      and its RMSE is measured on clean held-out pairs;
  (2) ordering: the predicate order by estimated cost (sum of exp(N) over the
      sample, N predicts the log of the cycles) against the order by the
      measured cost (sum of the measured cycles), as NDCG; the same for the
      library's 32-64-64-1 per-predicate model and for the rule- and
      data-aware plan's operation-count cost;
  (3) time: the measured cost of all sampled pairs (evaluating them) against
      the estimated cost (N's inference on their features).

Everything runs in libhb's kernels; this module draws the sample, splits it
and computes the metrics.

  python -m paper_2410_04349_gb300.model_study [--pairs N] [--epochs E]
"""
from __future__ import annotations

import json
import math
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))

from paper_2410_04349_gb300 import hb  # noqa: E402


def ndcg(true_cost, est_cost):
    """Order by ascending estimate against order by ascending true cost: the
    predicate at true rank r has relevance n - r; DCG = sum rel / log2(pos + 2)
    over the ideal DCG."""
    n = len(true_cost)
    rank_true = sorted(range(n), key=lambda i: (true_cost[i], i))
    rel = {p: n - r for r, p in enumerate(rank_true)}
    rank_est = sorted(range(n), key=lambda i: (est_cost[i], i))
    dcg = sum(rel[p] / math.log2(r + 2) for r, p in enumerate(rank_est))
    return dcg / sum(rel[p] / math.log2(r + 2) for r, p in enumerate(rank_true))


def study(table, mds, n_pairs=6000, betas=(0, 20, 40, 60, 80), epochs=1500, lr=1e-2, seed=0, model=None):
    rng = np.random.default_rng(seed)
    n = table.n_rows
    with hb.Context(device=0) as ctx:
        ctx.load_table(0, n, table.columns)
        for md in mds:
            ctx.add_md(md)
        info = ctx.plan("rule_data")
        preds = [int(p) for p in info.op_pred[:info.n_ops]]
        plain_cost = {p: info.cost[p] for p in preds}
        rows = {}
        t0 = time.perf_counter()
        for p in preds:
            i = rng.integers(0, n, n_pairs).astype(np.uint32)
            j = rng.integers(0, n, n_pairs).astype(np.uint32)
            cyc, ver, X = ctx.time_pairs(p, i, j)
            rows[p] = (X, np.log(np.maximum(cyc, 1)).astype(np.float32), cyc)
        exact_s = time.perf_counter() - t0
        learned_cost = None
        if model is not None:
            ctx.set_cost_model(model)
            li = ctx.plan("learned")
            learned_cost = {p: li.cost[p] for p in preds} if li.mode == 1 else None
    true_cost = [float(rows[p][2].sum()) for p in preds]
    split = int(0.7 * n_pairs)
    Xtr = np.concatenate([rows[p][0][:split] for p in preds])
    ytr = np.concatenate([rows[p][1][:split] for p in preds])
    Xte = np.concatenate([rows[p][0][split:] for p in preds])
    yte = np.concatenate([rows[p][1][split:] for p in preds])
    out = {"predicates": preds, "pairs_per_predicate": n_pairs, "train_rows": int(len(ytr)),
           "test_rows": int(len(yte)), "label": "ln(clock64 cycles) of checking the predicate on the pair",
           "noise": []}
    import torch
    dev_X = torch.from_numpy(np.concatenate([rows[p][0] for p in preds])).cuda()
    dev_y = torch.empty(dev_X.shape[0], device="cuda")
    dev_te = torch.from_numpy(Xte).cuda()
    y_te = torch.empty(dev_te.shape[0], device="cuda")
    for beta in betas:
        y_noisy = ytr.copy()
        k = int(round(len(y_noisy) * beta / 100.0))
        idx = rng.choice(len(y_noisy), size=k, replace=False)
        y_noisy[idx] = rng.uniform(ytr.min(), ytr.max(), size=k).astype(np.float32)
        params, train_mse = hb.train_pair_model(Xtr, y_noisy, epochs=epochs, lr=lr, seed=seed)
        dp = torch.from_numpy(params).cuda()
        hb.pair_model_forward(dev_te, dp, y_te)
        rmse = float(torch.sqrt(torch.mean((y_te.cpu() - torch.from_numpy(yte)) ** 2)))
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        hb.pair_model_forward(dev_X, dp, dev_y)
        torch.cuda.synchronize()
        est_s = time.perf_counter() - t1
        y_all = dev_y.cpu().numpy()
        est_cost, o = [], 0
        for p in preds:
            est_cost.append(float(np.exp(y_all[o:o + n_pairs].astype(np.float64)).sum()))
            o += n_pairs
        out["noise"].append({"beta_pct": beta, "test_rmse": rmse, "train_mse": float(train_mse),
                             "ndcg": ndcg(true_cost, est_cost), "estimate_s": est_s})
    out["exact_cost_s"] = exact_s
    out["ndcg_rule_data_cost"] = ndcg(true_cost, [plain_cost[p] for p in preds])
    if learned_cost is not None:
        out["ndcg_per_predicate_model"] = ndcg(true_cost, [learned_cost[p] for p in preds])
    return out


def main():
    import argparse
    import synth
    ap = argparse.ArgumentParser()
    ap.add_argument("--pairs", type=int, default=6000)
    ap.add_argument("--epochs", type=int, default=1500)
    ap.add_argument("--rows", type=int, default=200_000)
    args = ap.parse_args()
    t, mds = synth.config2(n=args.rows)
    model = np.load(os.path.join(HERE, "cost_model.npy")).astype(np.float32)
    print(json.dumps(study(t, mds, n_pairs=args.pairs, epochs=args.epochs, model=model)))


if __name__ == "__main__":
    main()
