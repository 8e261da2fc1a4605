"""Learned cost model: training with the library's kernels, predictions that
rank predicates better than the rule- and data-aware statistics, and a
learned plan that yields exactly the same pairs."""
import numpy as np
import pytest

import oracle
import synth
from paper_2410_04349_gb300 import hb, learn

pytestmark = pytest.mark.gpu


def _rows(ctx, t, sets):
    Xs, cs, ss = [], [], []
    ctx.load_table(0, t.n_rows, t.columns)
    for mds in sets:
        ctx.clear_mds()
        for md in mds:
            ctx.add_md(md)
        ctx.plan("rule_data")
        X, yc, ys = learn.collect(ctx)
        Xs.append(X)
        cs.append(yc)
        ss.append(ys)
    return np.concatenate(Xs), np.concatenate(cs), np.concatenate(ss)


def test_training_fits_and_learned_plan_is_exact():
    t, mds = synth.config2(n=60000, cards=(60, 600, 6000))
    sets = [mds] + [synth.random_rule_set(400 + i, 4, [2, 3, 4], [0, 1], [5, 6]) for i in range(6)]
    with hb.Context(device=0) as ctx:
        X, yc, ys = _rows(ctx, t, sets)
        assert X.shape[1] == hb.FEATURES and len(X) >= 20 and np.isfinite(X).all()
        loss = learn.train(ctx, X, yc, ys, epochs=800)
        assert loss[0] < 0.2 and loss[1] < 0.2          # standardized MSE on the training rows
        model = ctx.get_cost_model()
    # a held-out rule set on a held-out table
    t2, _ = synth.config2(seed=77, n=60000, cards=(60, 600, 6000))
    held = synth.random_rule_set(999, 4, [2, 3, 4], [0, 1], [5, 6])
    with hb.Context(device=0) as ctx:
        ctx.load_table(0, t2.n_rows, t2.columns)
        for md in held:
            ctx.add_md(md)
        ctx.set_cost_model(model)
        info_l = ctx.plan("learned")
        assert info_l.mode == 1
        got = ctx.block()
        info_p = ctx.plan("rule_data")
        want_gpu = ctx.block()
        logs = ctx.log_predicates(profile=True)
    want, _ = oracle.block_hash(t2, held)
    assert np.array_equal(got, want) and np.array_equal(want_gpu, want)
    # the network's selectivity ranks the measured pass rates better than sp of Section 4.2
    meas = {L["pred"]: L["passed"] / max(L["evaluated"], 1) for L in logs}
    ids = sorted(meas)
    if len(ids) >= 3:
        m = np.array([meas[i] for i in ids])
        pl = np.array([info_l.sp[i] for i in ids])
        pp = np.array([info_p.sp[i] for i in ids])
        rank = lambda a: np.argsort(np.argsort(a))
        corr = lambda a, b: np.corrcoef(rank(a), rank(b))[0, 1]
        assert corr(pl, m) >= corr(pp, m) - 1e-9


def test_learned_without_model_falls_back():
    t, mds = synth.config1()
    with hb.Context(device=0) as ctx:
        ctx.load_table(0, t.n_rows, t.columns)
        for md in mds:
            ctx.add_md(md)
        info = ctx.plan("learned")
        assert info.mode == 0            # rule- and data-aware plan applied
        with pytest.raises(hb.HBError):
            ctx.set_cost_model(np.full(2 * hb.MLP_PARAMS, np.nan, np.float32))


@pytest.mark.slow
def test_committed_model_gains_on_held_out_tables_and_rules():
    """The committed cost model (trained on logs of the 1M-tuple, R x S and batched
    workloads) against the rule- and data-aware plan on six held-out 3M-tuple
    tables of the 10M-tuple workload's schema, each with its own held-out set of
    16 rules: identical pair sets every time (one set also checked against the
    oracle on a 10 % row subset), and at least 1 % less evaluation time in all
    (CUDA events, median of 5 launches each)."""
    import statistics
    from fullsize_digest import c5_subset
    from gpu_helpers import committed_model
    model = committed_model()
    tot = {"rule_data": 0.0, "learned": 0.0}
    for s in range(6):
        t, _ = synth.config5(seed=synth.BASE_SEED + 500 + s, n=3_000_000)
        mds = synth.c5_mds(seed=synth.BASE_SEED + 700 + s)
        got = {}
        with hb.Context(device=0) as ctx:
            ctx.load_table(0, t.n_rows, t.columns)
            for md in mds:
                ctx.add_md(md)
            ctx.set_cost_model(model)
            for mode in ("rule_data", "learned"):
                info = ctx.plan(mode)
                assert info.mode == hb.PLAN_MODES[mode]
                for _ in range(2):
                    pairs = ctx.block()
                ev = []
                for _ in range(5):
                    pairs = ctx.block()
                    ev.append(ctx.stats()["ms_eval"])
                tot[mode] += statistics.median(ev)
                got[mode] = pairs
        assert np.array_equal(got["learned"], got["rule_data"])
        if s == 0:
            rows = c5_subset(t.n_rows, 1, 10)
            pos = np.full(t.n_rows, -1, np.int64)
            pos[rows] = np.arange(len(rows))
            a, b = pos[got["learned"][:, 0]], pos[got["learned"][:, 1]]
            keep = (a >= 0) & (b >= 0)
            sub = np.stack([a[keep], b[keep]], axis=1)
            sub = sub[np.lexsort((sub[:, 1], sub[:, 0]))]
            want, _ = oracle.block_owned(t.take(rows), mds)
            assert np.array_equal(sub, want)
    assert tot["learned"] <= 0.99 * tot["rule_data"], tot
