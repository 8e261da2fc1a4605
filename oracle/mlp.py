"""Cost-model MLP in fp64 numpy — TEST INFRASTRUCTURE ONLY.

The paper estimates predicate costs with a shallow feed-forward network N
trained offline on historical logs (Section 4.2, "Shallow NNs"; Section 6
uses ReLU and Adam).  The network built here has 32 inputs, two hidden ReLU
layers of 64 and one linear output:

    z1 = X W1 + b1,  h1 = relu(z1)
    z2 = h1 W2 + b2, h2 = relu(z2)
    y  = h2 W3 + b3
    loss = mean((y - t)^2)

Backward is the chain rule written out layer by layer; Adam follows Kingma &
Ba (2015), Algorithm 1, with bias correction.  ``forward_bf16`` is bf16
inference as this build specifies it: the inputs, the weights and each hidden
activation are rounded to bfloat16 (round to nearest even), the biases are
binary32, and products and sums are exact (fp64 here, at least fp32 on the
GPU); the output is not rounded.

Pinned in tests/test_oracle_mlp.py by closed forms (a network that sums its
inputs, a dead-ReLU network), central finite differences of the forward
function for every parameter, and the closed form of the first Adam step.
"""
from __future__ import annotations

import numpy as np

D_IN, H1, H2 = 32, 64, 64


def init_params(seed: int):
    """He-uniform initial weights (drawn with numpy's PCG64 from the seed)."""
    rng = np.random.Generator(np.random.PCG64(seed))

    def u(fan_in, shape):
        lim = np.sqrt(6.0 / fan_in)
        return rng.uniform(-lim, lim, size=shape)

    return {"W1": u(D_IN, (D_IN, H1)), "b1": np.zeros(H1), "W2": u(H1, (H1, H2)), "b2": np.zeros(H2),
            "W3": u(H2, (H2, 1)), "b3": np.zeros(1)}


def forward(p, X):
    X = np.asarray(X, np.float64)
    z1 = X @ p["W1"] + p["b1"]
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ p["W2"] + p["b2"]
    h2 = np.maximum(z2, 0.0)
    y = h2 @ p["W3"] + p["b3"]
    return y[:, 0], {"X": X, "z1": z1, "h1": h1, "z2": z2, "h2": h2}


def loss(p, X, t):
    y, _ = forward(p, X)
    return float(np.mean((y - np.asarray(t, np.float64)) ** 2))


def backward(p, X, t):
    """Gradients of the mean squared error with respect to every parameter."""
    y, c = forward(p, X)
    B = X.shape[0]
    dy = (2.0 / B) * (y - np.asarray(t, np.float64))[:, None]
    g = {}
    g["W3"] = c["h2"].T @ dy
    g["b3"] = dy.sum(axis=0)
    dh2 = dy @ p["W3"].T
    dz2 = dh2 * (c["z2"] > 0)
    g["W2"] = c["h1"].T @ dz2
    g["b2"] = dz2.sum(axis=0)
    dh1 = dz2 @ p["W2"].T
    dz1 = dh1 * (c["z1"] > 0)
    g["W1"] = c["X"].T @ dz1
    g["b1"] = dz1.sum(axis=0)
    return g


def adam_step(p, g, state, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update in place; state holds m, v and the step count t."""
    state["t"] = state.get("t", 0) + 1
    t = state["t"]
    for k in p:
        m = state.setdefault("m_" + k, np.zeros_like(p[k]))
        v = state.setdefault("v_" + k, np.zeros_like(p[k]))
        m[...] = beta1 * m + (1 - beta1) * g[k]
        v[...] = beta2 * v + (1 - beta2) * g[k] ** 2
        mhat = m / (1 - beta1 ** t)
        vhat = v / (1 - beta2 ** t)
        p[k] = p[k] - lr * mhat / (np.sqrt(vhat) + eps)
    return p


def to_bf16(x):
    """Round float values to the nearest bfloat16 (ties to even), returned as float64."""
    f = np.asarray(x, np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    rounded = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    nan = np.isnan(f)
    out = rounded.astype(np.uint32).view(np.float32).astype(np.float64)
    out[nan] = np.nan
    return out


def forward_bf16(p, X):
    """Inference with bf16 inputs, weights and hidden activations; sums in fp64,
    biases in fp32 precision."""
    Xb = to_bf16(X)
    W1, W2, W3 = to_bf16(p["W1"]), to_bf16(p["W2"]), to_bf16(p["W3"])
    b1 = np.asarray(p["b1"], np.float32).astype(np.float64)
    b2 = np.asarray(p["b2"], np.float32).astype(np.float64)
    b3 = np.asarray(p["b3"], np.float32).astype(np.float64)
    h1 = to_bf16(np.maximum(Xb @ W1 + b1, 0.0))
    h2 = to_bf16(np.maximum(h1 @ W2 + b2, 0.0))
    return (h2 @ W3 + b3)[:, 0]
