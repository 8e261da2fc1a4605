"""Cost model trained on the blocker's own logs (Section 4.2, "Shallow NNs":
a shallow feed-forward network estimates predicate costs and is trained
offline on historical logs).

``collect`` runs the current rules once with per-predicate instrumentation
(every predicate evaluated on every candidate pair, no early exit) and
returns one training row per non-equality predicate: its 32 features (kind,
threshold, sampled column statistics, rates measured on a row sample) and two
targets (log device cycles per evaluation, logit of the pass rate).
``train`` fits both networks on the GPU with the library's own forward,
backward and Adam kernels and installs them in the context, where
``plan("learned")`` uses them.  All computation happens in libhb.
"""
from __future__ import annotations

import numpy as np

from . import hb


def collect(ctx: "hb.Context"):
    """Training rows (features [n, 32], log_cost [n], logit_pass [n]) of the current rules."""
    logs = ctx.log_predicates(profile=True)
    rows = [L for L in logs if L["evaluated"] > 0]
    X = np.array([L["features"] for L in rows], np.float32).reshape(-1, hb.FEATURES)
    yc = np.array([L["log_cost"] for L in rows], np.float32)
    ys = np.array([L["logit_pass"] for L in rows], np.float32)
    return X, yc, ys


def train(ctx: "hb.Context", X, y_cost, y_sel, epochs=1500, lr=2e-3, seed=0):
    """Fit both networks and make them the context's model; returns the final
    training losses (standardized units)."""
    return ctx.train_cost_model(X, y_cost, y_sel, epochs=epochs, lr=lr, seed=seed)


def save(ctx: "hb.Context", path: str):
    np.save(path, ctx.get_cost_model())


def load(ctx: "hb.Context", path: str):
    ctx.set_cost_model(np.load(path))
