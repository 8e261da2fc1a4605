"""Shared helpers of the GPU tests: run libhb through its C-ABI binding."""
import numpy as np

from paper_2410_04349_gb300 import hb


def run_gpu(R, mds, S=None, mode="rule_data", tile=0, out_capacity=0, device_tables=False):
    with hb.Context(device=0, tile=tile, out_capacity=out_capacity) as ctx:
        ctx.load_table(0, R.n_rows, R.columns)
        if S is not None:
            ctx.load_table(1, S.n_rows, S.columns)
        for md in mds:
            ctx.add_md(md)
        info = ctx.plan(mode)
        pairs = ctx.block()
        st = ctx.stats()
    return pairs, st, info


def as_set(p):
    return set(map(tuple, np.asarray(p).tolist()))
