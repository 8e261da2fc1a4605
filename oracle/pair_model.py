"""The paper's per-pair cost model N in fp64 numpy — TEST INFRASTRUCTURE ONLY.

Section 4.2 ("Shallow NNs") estimates T_p(t1, t2), the time to check a
predicate p on a tuple pair, with a small feed-forward network N whose input
encodes p and the two tuples' A-values, trained offline on logged times; the
estimated cost of p is norm(sum of N(p, t1, t2) over (sampled) pairs).  The
experiments (Section 6, default parameters) use hidden layers of 2, 6 and 1
neurons with ReLU and Adam; this build reads that as the layer sizes
8 -> 2 -> 6 -> 1 over the 8 features below, ReLU after the first two, the
single last neuron being the output:

    z1 = x W1 + b1,  h1 = relu(z1)      (W1: 8 x 2)
    z2 = h1 W2 + b2, h2 = relu(z2)      (W2: 2 x 6)
    y  = h2 W3 + b3                     (W3: 6 x 1)

Features of (p, t1, t2) for an edit-distance, Jaccard or |a-b| predicate,
from the operand o of each tuple (string length for edit distance, the number
of distinct q-grams for Jaccard, the fp32 value for |a-b|):
    [ED?, JAC?, ABS?, threshold, s(o1), s(o2), s(|o1 - o2|), min/max]
with threshold = k/8, num/den or log1p(delta); s(v) = v/64 for lengths and
gram counts and log1p(|v|)/8 for values; min/max of |o1|, |o2| (0 when both
are 0); a missing operand sets features 4-7 to -1.

Pinned in tests/test_oracle_pair_model.py (central finite differences of the
forward function, a closed form, hand-computed features).
"""
from __future__ import annotations

import math

import numpy as np

SIZES = (8, 2, 6, 1)
N_PARAMS = 8 * 2 + 2 + 2 * 6 + 6 + 6 + 1


def unpack(theta):
    """Parameter dict from the flat layout W1, b1, W2, b2, W3, b3 (row-major)."""
    t = np.asarray(theta, np.float64)
    o = 0
    out = {}
    for name, shape in (("W1", (8, 2)), ("b1", (2,)), ("W2", (2, 6)), ("b2", (6,)), ("W3", (6, 1)), ("b3", (1,))):
        n = int(np.prod(shape))
        out[name] = t[o:o + n].reshape(shape)
        o += n
    return out


def pack(p):
    return np.concatenate([np.asarray(p[k], np.float64).ravel() for k in ("W1", "b1", "W2", "b2", "W3", "b3")])


def forward(p, X):
    X = np.asarray(X, np.float64)
    z1 = X @ p["W1"] + p["b1"]
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ p["W2"] + p["b2"]
    h2 = np.maximum(z2, 0.0)
    return (h2 @ p["W3"] + p["b3"])[:, 0], {"X": X, "z1": z1, "h1": h1, "z2": z2, "h2": h2}


def backward(p, X, t):
    """Gradients of mean((y - t)^2), layer by layer."""
    y, c = forward(p, X)
    dy = (2.0 / X.shape[0]) * (y - np.asarray(t, np.float64))[:, None]
    g = {"W3": c["h2"].T @ dy, "b3": dy.sum(axis=0)}
    dz2 = (dy @ p["W3"].T) * (c["z2"] > 0)
    g["W2"] = c["h1"].T @ dz2
    g["b2"] = dz2.sum(axis=0)
    dz1 = (dz2 @ p["W2"].T) * (c["z1"] > 0)
    g["W1"] = c["X"].T @ dz1
    g["b1"] = dz1.sum(axis=0)
    return g


def _grams(s: bytes, q: int) -> int:
    return len({s[i:i + q] for i in range(len(s) - q + 1)})


def features(pred, v1, v2):
    """The 8 inputs of N for predicate tuple pred and the two A-values (None = missing)."""
    kind = pred[0]
    f = [0.0] * 8
    if kind == "ed":
        f[0], f[3] = 1.0, pred[3] / 8.0
    elif kind == "jaccard":
        f[1], f[3] = 1.0, pred[5] / pred[6]
    elif kind == "absdiff":
        f[2], f[3] = 1.0, math.log1p(pred[7])
    else:
        raise ValueError(kind)
    if v1 is None or v2 is None:
        f[4:] = [-1.0] * 4
        return f
    if kind == "ed":
        o1, o2 = float(len(v1)), float(len(v2))
    elif kind == "jaccard":
        o1, o2 = float(_grams(v1, pred[4])), float(_grams(v2, pred[4]))
    else:
        o1, o2 = float(np.float32(v1)), float(np.float32(v2))
    if kind == "absdiff":
        s = lambda v: math.log1p(abs(v)) / 8.0
    else:
        s = lambda v: v / 64.0
    a1, a2 = abs(o1), abs(o2)
    f[4], f[5], f[6] = s(o1), s(o2), s(abs(o1 - o2))
    f[7] = min(a1, a2) / max(a1, a2) if max(a1, a2) > 0 else 0.0
    return f


def ndcg(true_cost, est_cost):
    """NDCG of the order by ascending estimated cost against the order by
    ascending true cost: the predicate ranked r-th (from 0) by true cost has
    relevance n - r; DCG = sum rel / log2(position + 2), over the ideal DCG."""
    n = len(true_cost)
    order_true = sorted(range(n), key=lambda i: (true_cost[i], i))
    rel = {p: n - r for r, p in enumerate(order_true)}
    order_est = sorted(range(n), key=lambda i: (est_cost[i], i))
    dcg = sum(rel[p] / math.log2(r + 2) for r, p in enumerate(order_est))
    idcg = sum(rel[p] / math.log2(r + 2) for r, p in enumerate(order_true))
    return dcg / idcg
