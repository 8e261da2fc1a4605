"""Pins of the fp64 MLP oracle: closed forms, finite differences, Adam."""
import numpy as np

from oracle import mlp


def test_forward_closed_form_sum_of_inputs():
    p = {"W1": np.zeros((32, 64)), "b1": np.zeros(64), "W2": np.zeros((64, 64)), "b2": np.zeros(64),
         "W3": np.zeros((64, 1)), "b3": np.array([0.5])}
    p["W1"][np.arange(32), np.arange(32)] = 1.0      # h1[:32] = relu(x)
    p["W2"][np.arange(32), np.arange(32)] = 1.0      # h2[:32] = h1[:32]
    p["W3"][:32, 0] = 1.0                             # y = sum relu(x) + 0.5
    X = np.random.default_rng(0).normal(size=(17, 32))
    y, _ = mlp.forward(p, X)
    assert np.allclose(y, np.maximum(X, 0).sum(axis=1) + 0.5, rtol=0, atol=1e-12)


def test_dead_relu_gives_bias_and_zero_grads():
    p = mlp.init_params(1)
    p["b1"][:] = -1e6
    X = np.random.default_rng(1).normal(size=(8, 32))
    y, _ = mlp.forward(p, X)
    assert np.allclose(y, p["b3"][0])
    g = mlp.backward(p, X, np.zeros(8))
    assert np.all(g["W1"] == 0) and np.all(g["W2"] == 0) and np.all(g["W3"] == 0)
    assert np.isclose(g["b3"][0], 2 * np.mean(y))


def test_backward_matches_central_differences():
    rng = np.random.default_rng(3)
    p = mlp.init_params(3)
    for k in p:
        p[k] = p[k] + rng.normal(scale=0.05, size=p[k].shape)
    X = rng.normal(size=(12, 32))
    t = rng.normal(size=12)
    g = mlp.backward(p, X, t)
    h = 1e-6
    for k in p:
        flat = p[k].reshape(-1)
        idx = rng.choice(flat.size, size=min(flat.size, 20), replace=False)
        for i in idx:
            old = flat[i]
            flat[i] = old + h
            lp = mlp.loss(p, X, t)
            flat[i] = old - h
            lm = mlp.loss(p, X, t)
            flat[i] = old
            num = (lp - lm) / (2 * h)
            assert abs(num - g[k].reshape(-1)[i]) <= 1e-6 + 1e-5 * abs(num), (k, i)


def test_first_adam_step_is_lr_times_sign():
    p = {"w": np.array([1.0, -2.0, 3.0])}
    g = {"w": np.array([0.5, -4.0, 1e-3])}
    st = {}
    mlp.adam_step(p, g, st, lr=0.01, eps=1e-12)
    assert np.allclose(p["w"], np.array([1.0 - 0.01, -2.0 + 0.01, 3.0 - 0.01]), atol=1e-9)


def test_training_reduces_loss_on_linear_target():
    rng = np.random.default_rng(4)
    X = rng.normal(size=(256, 32))
    t = X[:, :4].sum(axis=1)
    p = mlp.init_params(4)
    st = {}
    l0 = mlp.loss(p, X, t)
    for _ in range(300):
        mlp.adam_step(p, mlp.backward(p, X, t), st, lr=3e-3)
    assert mlp.loss(p, X, t) < 0.05 * l0


def test_bf16_rounding_ties_to_even():
    assert mlp.to_bf16(np.array([1.0]))[0] == 1.0
    # 1 + 2^-8 is a tie between 1 and 1 + 2^-7: even mantissa is 1.0
    assert mlp.to_bf16(np.array([1.0 + 2 ** -8]))[0] == 1.0
    assert mlp.to_bf16(np.array([1.0 + 3 * 2 ** -8]))[0] == 1.0 + 2 ** -6
    assert mlp.to_bf16(np.array([1.0 + 2 ** -8 + 2 ** -20]))[0] == 1.0 + 2 ** -7
