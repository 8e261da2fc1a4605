"""Host-side checks of the C-ABI library (no GPU needed): it loads, exports
every entry point the header declares, its host-only planner matches the plan
oracle, and calls fail cleanly (status + message) without a usable GPU."""
import os
import random
import re

import numpy as np
import pytest

import oracle.plan as OP
from paper_2410_04349_gb300 import hb

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "hb.h")).read()
    return sorted(set(re.findall(r"HB_API[^;(]*?\b(hb_\w+)\s*\(", text)))


def test_library_exports_every_declared_symbol():
    L = hb.lib()
    names = declared_symbols()
    assert len(names) >= 20
    for n in names:
        assert hasattr(L, n), n
    assert set(names) == set(hb.EXPORTS)


def test_version_string():
    assert b"sm_103a" in hb.lib().hb_version()


PAPER_MDS = [[0, 1, 2, 3], [2, 4], [5, 4]]
PAPER_SP = [1.0, 0.3, 0.4, 0.4, 0.2, 0.3]
PAPER_COST = [0.1, 0.2, 0.1, 0.6, 0.9, 0.5]


def test_plan_order_paper_example():
    prog, cp, order = hb.plan_order(PAPER_SP, PAPER_COST, PAPER_MDS)
    r = OP.plan(PAPER_MDS, PAPER_SP, PAPER_COST)
    seq, ocp = OP.flatten_program(r["path"], PAPER_MDS)
    assert order == r["md_order"] == [1, 0, 2]
    assert prog == seq and cp == ocp


def test_plan_order_matches_oracle_random():
    rng = random.Random(12)
    for _ in range(300):
        n_p = rng.randint(1, 16)
        mds = [rng.sample(range(n_p), rng.randint(1, min(6, n_p))) for _ in range(rng.randint(1, 10))]
        # coarse values make ties common, exercising the tie rules
        sp = [rng.choice([0.1, 0.2, 0.5, 1.0, rng.random()]) for _ in range(n_p)]
        cost = [rng.choice([0.1, 0.5, 1.0, rng.uniform(0.01, 1)]) for _ in range(n_p)]
        skip = [rng.random() < 0.3 for _ in range(n_p)]
        prog, cp, order = hb.plan_order(sp, cost, mds, skip)
        r = OP.plan(mds, sp, cost)
        seq, ocp = OP.flatten_program(r["path"], mds, skip={p for p in range(n_p) if skip[p]})
        assert order == r["md_order"]
        assert prog == seq
        assert cp == ocp


def test_plan_order_rejects_bad_input():
    with pytest.raises(hb.HBError):
        hb.plan_order([0.5], [0.0], [[0]])           # cost must be > 0
    with pytest.raises(hb.HBError):
        hb.plan_order([0.5], [1.0], [[3]])           # unknown predicate id


def test_create_without_gpu_fails_cleanly():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(hb.HBError) as e:
        hb.Context(device=0)
    assert e.value.status in (hb.HB_ERR_CUDA, hb.HB_ERR_ARG)
    assert "cuda" in str(e.value).lower()


def test_checked_library_exports_the_same_symbols():
    import ctypes
    path = os.path.join(ROOT, "paper_2410_04349_gb300", "libhb_checked.so")
    if not os.path.exists(path):
        pytest.skip("libhb_checked.so not built")
    L = ctypes.CDLL(path)
    for n in declared_symbols():
        assert hasattr(L, n), n
    L.hb_version.restype = ctypes.c_char_p
    assert b"checked" in L.hb_version()
    assert b"checked" not in hb.lib().hb_version()
