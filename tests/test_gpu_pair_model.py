"""GPU tests of the paper's per-pair cost model N (Section 4.2 "Shallow NNs",
8-2-6-1): the per-pair timing kernel's verdicts equal the oracle's single
predicate verdicts and its features equal the oracle's plain definition; the
network's forward pass and gradient equal the fp64 oracle; training fits; and
the Section 6 model study (noise -> RMSE, NDCG of the ordering, estimated vs
exact cost time) runs on the library's kernels."""
import numpy as np
import pytest

import oracle
import oracle.pair_model as pm
import synth
from paper_2410_04349_gb300 import hb

pytestmark = pytest.mark.gpu


def test_pair_times_verdicts_and_features_match_the_oracle():
    t, mds = synth.config2(n=5000, cards=(10, 100, 1000))
    rng = np.random.default_rng(1)
    i = rng.integers(0, t.n_rows, 3000).astype(np.uint32)
    j = rng.integers(0, t.n_rows, 3000).astype(np.uint32)
    with hb.Context(device=0) as ctx:
        ctx.load_table(0, t.n_rows, t.columns)
        for md in mds:
            ctx.add_md(md)
        info = ctx.plan("rule_data")
        dp = oracle.distinct_predicates(mds)
        for p in info.op_pred[:info.n_ops]:
            cyc, ver, X = ctx.time_pairs(int(p), i, j)
            pred = dp[int(p)]
            want = oracle.pred_verdicts(t, pred, np.stack([i, j], axis=1))
            assert np.array_equal(ver, want), pred
            assert (cyc > 0).all()
            col = t.columns[pred[1]]
            for k in range(0, 3000, 97):
                f = pm.features(pred, col.value(int(i[k])), col.value(int(j[k])))
                assert np.allclose(X[k], f, atol=1e-6), (pred, k)


def test_forward_and_gradient_match_the_fp64_oracle():
    import torch
    rng = np.random.default_rng(2)
    theta = rng.normal(0, 0.6, hb.PAIR_MODEL_PARAMS).astype(np.float32)
    X = rng.normal(0, 1, (1000, 8)).astype(np.float32)
    tgt = rng.normal(0, 1, 1000).astype(np.float32)
    dX, dt, dp = (torch.from_numpy(a).cuda() for a in (X, tgt, theta))
    y = torch.empty(1000, device="cuda")
    g = torch.empty(hb.PAIR_MODEL_PARAMS, device="cuda")
    hb.pair_model_forward(dX, dp, y)
    hb.pair_model_backward(dX, dt, dp, g)
    torch.cuda.synchronize()
    p = pm.unpack(theta.astype(np.float64))
    want_y, _ = pm.forward(p, X)
    want_g = pm.pack(pm.backward(p, X, tgt))
    assert np.allclose(y.cpu().numpy(), want_y, rtol=1e-4, atol=1e-5)
    assert np.allclose(g.cpu().numpy(), want_g, rtol=1e-3, atol=1e-5)


def test_training_fits_a_function_the_network_can_represent():
    rng = np.random.default_rng(3)
    X = rng.uniform(-1, 1, (4000, 8)).astype(np.float32)
    y = (1.5 * np.maximum(X[:, 0] + X[:, 3], 0) + 0.5).astype(np.float32)
    params, mse = hb.train_pair_model(X, y, epochs=3000, lr=1e-2, seed=5)
    assert mse < 0.05 * float(np.var(y)), mse
    assert np.isfinite(params).all()


@pytest.mark.slow
def test_model_study_runs_on_the_benchmark_rules():
    from gpu_helpers import committed_model
    from paper_2410_04349_gb300 import model_study
    t, mds = synth.config2(n=100_000)
    r = model_study.study(t, mds, n_pairs=3000, betas=(0, 40, 80), epochs=1000, model=committed_model())
    rm = [x["test_rmse"] for x in r["noise"]]
    assert rm[0] < rm[-1]                       # heavy label noise costs accuracy
    assert all(0 < x["ndcg"] <= 1 for x in r["noise"])
    assert 0 < r["ndcg_rule_data_cost"] <= 1 and 0 < r["ndcg_per_predicate_model"] <= 1
    # the study's NDCG equals the oracle's definition
    assert abs(model_study.ndcg([3, 1, 2], [2, 1, 3]) - pm.ndcg([3, 1, 2], [2, 1, 3])) < 1e-12
