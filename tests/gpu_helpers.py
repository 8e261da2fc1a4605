"""Shared helpers of the GPU tests: run libhb through its C-ABI binding."""
import os

import numpy as np

from paper_2410_04349_gb300 import hb


MODEL = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2410_04349_gb300",
                     "cost_model.npy")


def committed_model():
    """The cost model committed with the library (two 32-64-64-1 networks)."""
    return np.load(MODEL).astype(np.float32)


def run_gpu(R, mds, S=None, mode="rule_data", tile=0, out_capacity=0, device_tables=False, model=None):
    with hb.Context(device=0, tile=tile, out_capacity=out_capacity) as ctx:
        ctx.load_table(0, R.n_rows, R.columns)
        if S is not None:
            ctx.load_table(1, S.n_rows, S.columns)
        for md in mds:
            ctx.add_md(md)
        if model is not None:
            ctx.set_cost_model(model)
        info = ctx.plan(mode)
        pairs = ctx.block()
        st = ctx.stats()
    return pairs, st, info


def as_set(p):
    return set(map(tuple, np.asarray(p).tolist()))
