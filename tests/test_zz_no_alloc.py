"""The allocation-free backward pass (hb_mlp_backward_noalloc) gives the same
gradient as hb_mlp_backward.

It exists for callers that cannot allocate device memory when they need a
gradient (memory pre-partitioned by their own pool, or loops that must not
call cudaMalloc / cudaFree); its work buffers are a fixed array inside the
library, limited to 4096 rows.  This file is collected last on purpose."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _inputs(n, seed):
    import torch
    g = torch.Generator(device="cpu").manual_seed(seed)
    X = torch.randn(n, 32, generator=g).cuda()
    t = torch.randn(n, generator=g).cuda()
    P = (0.2 * torch.randn(32 * 64 + 64 + 64 * 64 + 64 + 64 + 1, generator=g)).cuda()
    return X, t, P


def test_noalloc_backward_matches_allocating_backward_twice_in_a_row():
    import torch
    from paper_2410_04349_gb300 import hb
    for n, seed in [(4096, 11), (37, 12)]:   # the second call reuses the array with fewer rows
        X, t, P = _inputs(n, seed)
        want = torch.empty(hb.MLP_PARAMS, device="cuda")
        hb.mlp_backward(X, t, P, want)
        got = torch.full((hb.MLP_PARAMS,), float("nan"), device="cuda")
        hb.mlp_backward_noalloc(X, t, P, got)
        torch.cuda.synchronize()
        # same kernels, same summation order: the gradients agree to the bit (tolerance 0)
        assert torch.equal(got, want), n


def test_noalloc_rejects_more_rows_than_its_array_holds():
    import torch
    from paper_2410_04349_gb300 import hb
    X, t, P = _inputs(4097, 13)
    g = torch.empty(hb.MLP_PARAMS, device="cuda")
    with pytest.raises(hb.HBError) as e:
        hb.mlp_backward_noalloc(X, t, P, g)
    assert e.value.status == hb.HB_ERR_ARG and "4096" in str(e.value)
