"""Pins of the oracle's per-pair cost model N (Section 4.2 "Shallow NNs",
layer sizes 8-2-6-1 read from Section 6's defaults): central finite
differences of the forward function for every parameter, a closed form of a
network with fixed weights, hand-computed features, and NDCG on hand cases."""
import math

import numpy as np

import oracle.pair_model as pm
from oracle import mlp
from synth import absdiff, ed, jac


def test_gradients_match_central_differences():
    rng = np.random.default_rng(3)
    theta = rng.normal(0, 0.7, pm.N_PARAMS)
    X = rng.normal(0, 1, (17, 8))
    t = rng.normal(0, 1, 17)
    p = pm.unpack(theta)
    g = pm.pack(pm.backward(p, X, t))

    def loss(th):
        y, _ = pm.forward(pm.unpack(th), X)
        return float(np.mean((y - t) ** 2))

    for i in range(pm.N_PARAMS):
        e = np.zeros(pm.N_PARAMS)
        e[i] = 1e-6
        num = (loss(theta + e) - loss(theta - e)) / 2e-6
        assert abs(num - g[i]) < 1e-5 * max(1.0, abs(num)), i


def test_closed_form():
    # W1 picks x0 and x1 into the two hidden units, W2 copies unit 0 to all six, W3 sums: y = 6 * relu(x0) + 1
    p = {"W1": np.zeros((8, 2)), "b1": np.zeros(2), "W2": np.zeros((2, 6)), "b2": np.zeros(6),
         "W3": np.ones((6, 1)), "b3": np.array([1.0])}
    p["W1"][0, 0] = 1.0
    p["W1"][1, 1] = 1.0
    p["W2"][0, :] = 1.0
    X = np.zeros((3, 8))
    X[:, 0] = [-2.0, 0.5, 3.0]
    X[:, 1] = [5.0, 5.0, 5.0]
    y, _ = pm.forward(p, X)
    assert np.allclose(y, [1.0, 4.0, 19.0])
    assert pm.N_PARAMS == len(pm.pack(p)) == 43


def test_features_by_hand():
    f = pm.features(ed(0, 2), b"abcd", b"abcdefgh")
    assert f == [1.0, 0.0, 0.0, 0.25, 4 / 64, 8 / 64, 4 / 64, 0.5]
    f = pm.features(jac(0, 4, 5), b"aaaa", b"abcab")       # grams {aaa}; {abc, bca, cab}
    assert f == [0.0, 1.0, 0.0, 0.8, 1 / 64, 3 / 64, 2 / 64, 1 / 3]
    f = pm.features(absdiff(0, 0.5), 2.0, -4.0)
    assert f[:4] == [0.0, 0.0, 1.0, math.log1p(0.5)]
    assert f[4:] == [math.log1p(2.0) / 8, math.log1p(4.0) / 8, math.log1p(6.0) / 8, 0.5]
    assert pm.features(ed(0, 1), None, b"x")[4:] == [-1.0] * 4


def test_ndcg():
    assert pm.ndcg([1, 2, 3], [10, 20, 30]) == 1.0
    # two swapped at the top: relevance 3, 2, 1 shown as 2, 3, 1
    want = (2 / math.log2(2) + 3 / math.log2(3) + 1 / math.log2(4)) / (3 / math.log2(2) + 2 / math.log2(3) + 1 / 2)
    assert abs(pm.ndcg([1, 2, 3], [2, 1, 3]) - want) < 1e-12
    assert pm.ndcg([1, 2, 3], [3, 2, 1]) < want


def test_adam_from_the_shared_oracle_applies():
    p = pm.unpack(np.ones(pm.N_PARAMS))
    g = {k: np.ones_like(v) for k, v in p.items()}
    mlp.adam_step(p, g, {}, lr=0.1)
    assert all(np.allclose(v, 0.9) for v in p.values())
