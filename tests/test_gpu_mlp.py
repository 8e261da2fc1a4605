"""Cost-model MLP kernels (C-ABI) against the fp64 oracle."""
import numpy as np
import pytest

from oracle import mlp as M

pytestmark = pytest.mark.gpu


def flat(p):
    return np.concatenate([p["W1"].ravel(), p["b1"], p["W2"].ravel(), p["b2"], p["W3"].ravel(), p["b3"]])


def unflat(v):
    o = 0
    p = {}
    for k, shape in [("W1", (32, 64)), ("b1", (64,)), ("W2", (64, 64)), ("b2", (64,)), ("W3", (64, 1)), ("b3", (1,))]:
        n = int(np.prod(shape))
        p[k] = np.asarray(v[o:o + n], np.float64).reshape(shape)
        o += n
    return p


def setup(n, seed):
    import torch
    rng = np.random.default_rng(seed)
    p = M.init_params(seed)
    for k in p:
        p[k] = p[k] + rng.normal(scale=0.05, size=p[k].shape)
    X = rng.normal(size=(n, 32))
    t = rng.normal(size=n)
    dev = torch.device("cuda")
    Xd = torch.tensor(X, dtype=torch.float32, device=dev)
    td = torch.tensor(t, dtype=torch.float32, device=dev)
    Pd = torch.tensor(flat(p), dtype=torch.float32, device=dev)
    # the oracle sees exactly the fp32 values the GPU sees
    p32 = unflat(flat(p).astype(np.float32).astype(np.float64))
    return p32, X.astype(np.float32).astype(np.float64), t.astype(np.float32).astype(np.float64), Xd, td, Pd


@pytest.mark.parametrize("n", [1, 31, 32, 33, 1000])
def test_forward_fp32(n):
    import torch
    from paper_2410_04349_gb300 import hb
    p, X, t, Xd, td, Pd = setup(n, 1)
    y = torch.empty(n, dtype=torch.float32, device="cuda")
    hb.mlp_forward(Xd, Pd, y)
    want, _ = M.forward(p, X)
    got = y.cpu().numpy().astype(np.float64)
    # fp32 accumulation over at most 65 terms per unit: relative 1e-5 of the term magnitudes
    assert np.allclose(got, want, rtol=1e-4, atol=1e-4 * (1 + np.abs(want).max()))


def test_forward_bf16_matches_emulated_rounding():
    import torch
    from paper_2410_04349_gb300 import hb
    n = 777
    p, X, t, Xd, td, Pd = setup(n, 2)
    y = torch.empty(n, dtype=torch.float32, device="cuda")
    hb.mlp_forward(Xd, Pd, y, bf16=True)
    want = M.forward_bf16(p, X)
    got = y.cpu().numpy().astype(np.float64)
    # fp32 vs fp64 sums can round a hidden activation to the neighbouring bf16 value (2^-8 relative);
    # the bound allows a few such flips per output
    scale = 1 + np.abs(want).max()
    assert np.max(np.abs(got - want)) <= 2 ** -6 * scale
    assert np.mean(np.abs(got - want)) <= 2 ** -10 * scale
    full, _ = M.forward(p, X)
    assert np.max(np.abs(got - full)) <= 0.05 * scale


@pytest.mark.parametrize("n", [1, 64, 1000])
def test_backward_matches_oracle(n):
    import torch
    from paper_2410_04349_gb300 import hb
    p, X, t, Xd, td, Pd = setup(n, 3)
    g = torch.empty(hb.MLP_PARAMS, dtype=torch.float32, device="cuda")
    hb.mlp_backward(Xd, td, Pd, g)
    want = flat(M.backward(p, X, t))
    got = g.cpu().numpy().astype(np.float64)
    assert np.allclose(got, want, rtol=1e-3, atol=1e-5 * (1 + np.abs(want).max()))


def test_adam_step_matches_oracle():
    import torch
    from paper_2410_04349_gb300 import hb
    rng = np.random.default_rng(4)
    n = hb.MLP_PARAMS
    w = rng.normal(size=n).astype(np.float32)
    g1 = rng.normal(size=n).astype(np.float32)
    g2 = rng.normal(size=n).astype(np.float32)
    wd = torch.tensor(w, device="cuda")
    md = torch.zeros(n, device="cuda")
    vd = torch.zeros(n, device="cuda")
    p = {"w": w.astype(np.float64)}
    st = {}
    for step, g in enumerate([g1, g2], start=1):
        hb.adam_step(wd, torch.tensor(g, device="cuda"), md, vd, step, lr=1e-2)
        M.adam_step(p, {"w": g.astype(np.float64)}, st, lr=1e-2)
    assert np.allclose(wd.cpu().numpy(), p["w"], rtol=0, atol=1e-6)
