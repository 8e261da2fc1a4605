"""CPU oracle for rule-based blocking — TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The GPU library and its Python binding
never import it, and it imports nothing from them.

Contents:
  * hb_oracle.cpp   - the blocking definition of Section 2 ("Semantics",
                      "Blocking") as a literal nested loop, a grouped variant,
                      per-pair checks, the single predicates and an
                      owner-rule pass for the benchmark's full sizes;
  * plan.py         - the execution-plan generator of Section 4.2 (ordering by
                      cost-effectiveness, execution tree, witness probability,
                      edge scores, DFS order) and its flattening into the
                      sequential execution path of Section 5.1;
  * mlp.py          - fp64 forward / backward / Adam for the cost-model MLP.

This module marshals numpy tables (see ``synth``) into the C oracle.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")

KINDS = {"eq": 0, "eq_prefix": 1, "ed": 2, "jaccard": 3, "absdiff": 4, "const_eq": 5, "contain": 6, "tjaccard": 7}


class OrCol(ctypes.Structure):
    _fields_ = [("type", ctypes.c_int32), ("pad", ctypes.c_int32), ("data", ctypes.c_void_p),
                ("off", ctypes.c_void_p), ("valid", ctypes.c_void_p)]


class OrPred(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("col_t", ctypes.c_int32), ("col_s", ctypes.c_int32),
                ("k", ctypes.c_int32), ("q", ctypes.c_int32), ("num", ctypes.c_uint32), ("den", ctypes.c_uint32),
                ("delta", ctypes.c_float), ("side", ctypes.c_int32), ("value_len", ctypes.c_uint32),
                ("value", ctypes.c_void_p)]


_CONSTS = []   # constant bytes referenced by marshalled predicates (kept alive)


def _const_bytes(v):
    """A constant as the oracle reads it: bytes of a string, or an int32's 4 bytes."""
    if isinstance(v, (bytes, bytearray, str)):
        b = v.encode() if isinstance(v, str) else bytes(v)
    else:
        b = np.array([v], np.int32).tobytes()
    buf = ctypes.create_string_buffer(b, max(len(b), 1))
    _CONSTS.append(buf)
    return buf, len(b)


def build(force: bool = False) -> str:
    """Compile liboracle.so (plain C++17, -O2, no fast-math, no contraction)."""
    src = os.path.join(_HERE, "hb_oracle.cpp")
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fno-fast-math", "-shared",
                               "-fPIC", "-pthread", "-o", tmp, src])
        os.replace(tmp, _SO)
    return _SO


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_SO)
        P = ctypes.c_void_p
        i64, i32 = ctypes.c_int64, ctypes.c_int32
        L.or_edit_distance.restype = i64
        L.or_edit_distance.argtypes = [P, i64, P, i64]
        L.or_qgram_sets.restype = None
        L.or_qgram_sets.argtypes = [P, i64, P, i64, i32, P, P, P]
        L.or_jaccard_ge.restype = i32
        L.or_jaccard_ge.argtypes = [P, i64, P, i64, i32, ctypes.c_uint32, ctypes.c_uint32]
        L.or_absdiff_le.restype = i32
        L.or_absdiff_le.argtypes = [ctypes.c_float, ctypes.c_float, ctypes.c_float]
        L.or_block_literal.restype = i64
        L.or_block_literal.argtypes = [i64, i32, P, i64, i32, P, i32, P, P, P, i64]
        L.or_block_hash.restype = i64
        L.or_block_hash.argtypes = [i64, i32, P, i64, i32, P, i32, P, P, i32, P, i64, P, i32]
        L.or_block_owned.restype = i64
        L.or_block_owned.argtypes = [i64, i32, P, i64, i32, P, i32, P, P, i32, i32, P, i64, P]
        L.or_plan_units.restype = i64
        L.or_plan_units.argtypes = [i64, i32, P, i64, i32, P, i32, P, P, i32, i32, i32, P, P, P, P]
        L.or_check_pairs.restype = None
        L.or_check_pairs.argtypes = [i64, i32, P, i64, i32, P, i32, P, P, P, i64, P]
        L.or_pred_verdicts.restype = None
        L.or_pred_verdicts.argtypes = [i64, i32, P, i64, i32, P, P, P, i64, P]
        _lib = L
    return _lib


def _buf(b: bytes | bytearray | str):
    if isinstance(b, str):
        b = b.encode()
    a = np.frombuffer(bytes(b), np.uint8) if len(b) else np.zeros(1, np.uint8)
    return a, len(b)


def edit_distance(a, b) -> int:
    A, la = _buf(a)
    B, lb = _buf(b)
    return int(lib().or_edit_distance(A.ctypes.data, la, B.ctypes.data, lb))


def qgram_sets(a, b, q=3):
    A, la = _buf(a)
    B, lb = _buf(b)
    out = np.zeros(3, np.int64)
    lib().or_qgram_sets(A.ctypes.data, la, B.ctypes.data, lb, q, out.ctypes.data, out[1:].ctypes.data,
                        out[2:].ctypes.data)
    return int(out[0]), int(out[1]), int(out[2])


def jaccard_ge(a, b, num, den, q=3) -> bool:
    A, la = _buf(a)
    B, lb = _buf(b)
    return bool(lib().or_jaccard_ge(A.ctypes.data, la, B.ctypes.data, lb, q, num, den))


def absdiff_le(a: float, b: float, delta: float) -> bool:
    return bool(lib().or_absdiff_le(a, b, delta))


class _Marshal:
    """Keeps numpy buffers alive while the C oracle reads them."""

    def __init__(self, table):
        self.keep = []
        n = len(table.columns)
        self.arr = (OrCol * max(n, 1))()
        for i, c in enumerate(table.columns):
            col = OrCol()
            col.type = {"string": 0, "int32": 1, "fp32": 2}[c.type]
            data = c.data if len(c.data) else np.zeros(1, c.data.dtype)
            self.keep.append(data)
            col.data = data.ctypes.data
            if c.offsets is not None:
                off = np.ascontiguousarray(c.offsets, np.uint32)
                self.keep.append(off)
                col.off = off.ctypes.data
            if c.valid is not None:
                v = np.ascontiguousarray(c.valid, np.uint8)
                self.keep.append(v)
                col.valid = v.ctypes.data
            self.arr[i] = col
        self.n = table.n_rows
        self.ncols = n


def _rules(mds):
    starts = np.zeros(len(mds) + 1, np.int32)
    flat = []
    for m, preds in enumerate(mds):
        flat.extend(preds)
        starts[m + 1] = len(flat)
    arr = (OrPred * max(len(flat), 1))()
    for i, p in enumerate(flat):
        kind, ct, cs, k, q, num, den, delta = p[:8]
        side = p[8] if len(p) > 8 else 0
        op = OrPred(KINDS[kind], ct, cs, k, q, num, den, delta, side, 0, None)
        if kind == "const_eq":
            buf, n = _const_bytes(p[9])
            op.value = ctypes.cast(buf, ctypes.c_void_p)
            op.value_len = n
        arr[i] = op
    return starts, arr


def _args(R, S):
    r = _Marshal(R)
    s = _Marshal(S) if S is not None else None
    return r, s, (r.n, r.ncols, r.arr, s.n if s else 0, s.ncols if s else 0, s.arr if s else None)


def _unpack(buf, n):
    v = buf[:n]
    return np.stack([(v >> 32).astype(np.int64), (v & 0xFFFFFFFF).astype(np.int64)], axis=1) if n else \
        np.zeros((0, 2), np.int64)


def block_literal(R, mds, S=None) -> np.ndarray:
    """Pairs (i, j) of the naive nested loop, ascending; shape [n, 2]."""
    r, s, a = _args(R, S)
    starts, preds = _rules(mds)
    n = lib().or_block_literal(*a, len(mds), starts.ctypes.data, preds, None, 0)
    buf = np.zeros(max(n, 1), np.uint64)
    lib().or_block_literal(*a, len(mds), starts.ctypes.data, preds, buf.ctypes.data, n)
    return _unpack(buf, n)


def block_hash(R, mds, S=None, threads=None, count_candidates=True):
    """(pairs [n,2] ascending, candidate count) of the grouped evaluation."""
    r, s, a = _args(R, S)
    starts, preds = _rules(mds)
    threads = threads or os.cpu_count() or 1
    cand = np.zeros(1, np.int64)
    n = lib().or_block_hash(*a, len(mds), starts.ctypes.data, preds, threads, None, 0, cand.ctypes.data,
                            1 if count_candidates else 0)
    buf = np.zeros(max(n, 1), np.uint64)
    lib().or_block_hash(*a, len(mds), starts.ctypes.data, preds, threads, buf.ctypes.data, n, None, 0)
    return _unpack(buf, n), int(cand[0])


def block_owned(R, mds, S=None, threads=None, evaluate=True):
    """(pairs [n,2] ascending, candidate count) by the owner rule: each pair
    that agrees on some MD's equality predicates is looked at once, in the
    group of the lowest such MD; for relations of the benchmark's full sizes.
    evaluate=False only counts the candidates (pairs is then empty)."""
    r, s, a = _args(R, S)
    starts, preds = _rules(mds)
    threads = threads or os.cpu_count() or 1
    cand = np.zeros(1, np.int64)
    if not evaluate:
        lib().or_block_owned(*a, len(mds), starts.ctypes.data, preds, threads, 0, None, 0, cand.ctypes.data)
        return np.zeros((0, 2), np.int64), int(cand[0])
    # one pass: the result is written into a buffer grown until it fits
    cap = 1 << 20
    while True:
        buf = np.zeros(cap, np.uint64)
        n = lib().or_block_owned(*a, len(mds), starts.ctypes.data, preds, threads, 1, buf.ctypes.data, cap,
                                 cand.ctypes.data)
        if n <= cap:
            return _unpack(buf, n), int(cand[0])
        cap = int(n)


def _norm_pred(p):
    """A predicate with only the parameters its kind uses (a Jaccard threshold
    as a reduced fraction): two predicates are the same iff these are equal."""
    kind, ct, cs, k, q, num, den, delta = p[:8]
    side = p[8] if len(p) > 8 else 0
    if kind == "const_eq":
        return (kind, ct, cs, side, p[9])
    if kind == "contain":
        from math import gcd
        g = gcd(num, den) or 1
        return (kind, ct, cs, q, num // g, den // g, side)
    if kind == "tjaccard":
        from math import gcd
        g = gcd(num, den) or 1
        return (kind, ct, cs, num // g, den // g)
    if kind == "eq":
        return (kind, ct, cs)
    if kind in ("eq_prefix", "ed"):
        return (kind, ct, cs, k)
    if kind == "jaccard":
        from math import gcd
        g = gcd(num, den) or 1
        return (kind, ct, cs, q, num // g, den // g)
    return (kind, ct, cs, float(np.float32(delta)))


def distinct_predicates(mds):
    """Distinct predicates in order of first appearance over the MDs (MD order,
    then written order): the numbering of Section 4.2's per-predicate
    quantities and of the plan's program."""
    out = []
    for md in mds:
        for p in md:
            if _norm_pred(p) not in [_norm_pred(x) for x in out]:
                out.append(p)
    return out


UNIT_NAMES = ("eq", "owner", "absdiff", "ed", "jaccard")


def plan_units(R, mds, program, S=None, threads=None):
    """Algorithmic work of replaying a plan on every candidate pair: a dict of
    units per class (see or_plan_units), 'candidates', and 'total'.  program
    lists the distinct non-equality predicates (tuples) in plan order."""
    r, s, a = _args(R, S)
    starts, preds = _rules(mds)
    flat = [p for md in mds for p in md]
    key = [_norm_pred(p) for p in flat]
    prog, need = [], []
    for p in program:
        kp = _norm_pred(p)
        prog.append(key.index(kp))
        need.append(sum(1 << m for m, md in enumerate(mds) if any(_norm_pred(x) == kp for x in md)))
    cp = []
    for md in mds:
        steps = [i for i, p in enumerate(program) if any(_norm_pred(x) == _norm_pred(p) for x in md)]
        others = [x for x in md if x[0] not in ("eq", "eq_prefix")]
        if len({_norm_pred(x) for x in others}) != len(steps):
            raise ValueError("program misses a non-equality predicate of an MD")
        cp.append(max(steps, default=-1))
    n_eq = len({_norm_pred(x) for x in flat if x[0] in ("eq", "eq_prefix")})
    prog_a = np.array(prog or [0], np.int32)
    need_a = np.array(need or [0], np.uint64)
    cp_a = np.array(cp, np.int32)
    out = np.zeros(7, np.int64)
    threads = threads or os.cpu_count() or 1
    lib().or_plan_units(*a, len(mds), starts.ctypes.data, preds, threads, n_eq, len(prog), prog_a.ctypes.data,
                        need_a.ctypes.data, cp_a.ctypes.data, out.ctypes.data)
    if out[6]:
        raise AssertionError(f"plan replay disagrees with the disjunction on {out[6]} pairs")
    d = {n: int(v) for n, v in zip(UNIT_NAMES, out[:5])}
    d["candidates"] = int(out[5])
    d["total"] = int(out[:5].sum())
    return d


def check_pairs(R, mds, pairs, S=None) -> np.ndarray:
    """Verdict (0/1) of the disjunction for each given pair (i, j)."""
    r, s, a = _args(R, S)
    starts, preds = _rules(mds)
    pairs = np.asarray(pairs, np.int64).reshape(-1, 2)
    packed = ((pairs[:, 0].astype(np.uint64) << np.uint64(32)) | pairs[:, 1].astype(np.uint64)).copy()
    out = np.zeros(max(len(packed), 1), np.uint8)
    lib().or_check_pairs(*a, len(mds), starts.ctypes.data, preds, packed.ctypes.data, len(packed), out.ctypes.data)
    return out[:len(packed)]


def pred_verdicts(R, pred, pairs, S=None) -> np.ndarray:
    """Verdict (0/1) of one predicate for each given pair (i, j)."""
    r, s, a = _args(R, S)
    _, preds = _rules([[pred]])
    pairs = np.asarray(pairs, np.int64).reshape(-1, 2)
    packed = ((pairs[:, 0].astype(np.uint64) << np.uint64(32)) | pairs[:, 1].astype(np.uint64)).copy()
    out = np.zeros(max(len(packed), 1), np.uint8)
    lib().or_pred_verdicts(*a, preds, packed.ctypes.data, len(packed), out.ctypes.data)
    return out[:len(packed)]
