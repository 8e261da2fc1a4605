"""Seeded synthetic relations and rule sets for the blocking workloads.

This module is shared by the CPU oracle's tests and by the GPU library's
tests and benchmark.  It creates input data only (columns, near-duplicates,
job layouts, rule lists); it contains no part of the blocking method itself.

Workload shapes follow the paper's experimental setting (Section 6: relations
of 10^3..10^7 tuples with string, categorical and numeric attributes, a few
to tens of MDs of up to ten predicates).  The paper's own datasets are not
available; these seeded tables stand in for them.

Column representation (numpy, host memory):
  string : data uint8[nbytes], offsets uint32[n+1]
  int32  : data int32[n]
  fp32   : data float32[n]
  valid  : uint8[n] (1 = present) or None (all present)

Predicate representation: a tuple ``(kind, col_t, col_s, k, q, num, den, delta[, side[, value]])``
with kind one of "eq", "eq_prefix", "ed", "jaccard", "absdiff", "const_eq", "contain",
"tjaccard" (side and value as in ``const_eq`` / ``contain``).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "libsynth.so")

LETTERS, WORDS, ZIPF_INT, ZIPF_STR, UNIFORM_INT, UNIFORM_STR, LOGNORMAL, ROWID = range(8)


class _ColSpec(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("lo", ctypes.c_int32), ("hi", ctypes.c_int32),
                ("card", ctypes.c_int64), ("zipf_s", ctypes.c_double), ("mu", ctypes.c_double),
                ("sigma", ctypes.c_double), ("null_rate", ctypes.c_double), ("edit", ctypes.c_int32),
                ("pad", ctypes.c_int32)]


class _TableSpec(ctypes.Structure):
    _fields_ = [("n_rows", ctypes.c_int64), ("dup_rate", ctypes.c_double), ("cross_rate", ctypes.c_double),
                ("edit_lo", ctypes.c_int32), ("edit_hi", ctypes.c_int32), ("swap_p", ctypes.c_double),
                ("noise_rel", ctypes.c_double), ("seed", ctypes.c_uint64), ("n_cols", ctypes.c_int32),
                ("shuffle", ctypes.c_int32)]


class _Col(ctypes.Structure):
    _fields_ = [("type", ctypes.c_int32), ("pad", ctypes.c_int32), ("n", ctypes.c_int64),
                ("bytes", ctypes.POINTER(ctypes.c_uint8)), ("nbytes", ctypes.c_uint64),
                ("off", ctypes.POINTER(ctypes.c_uint32)), ("i32", ctypes.POINTER(ctypes.c_int32)),
                ("f32", ctypes.POINTER(ctypes.c_float)), ("valid", ctypes.POINTER(ctypes.c_uint8))]


def build(force: bool = False) -> str:
    """Compile libsynth.so next to this file (plain C, no GPU code)."""
    src = os.path.join(_HERE, "synth.c")
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp, src, "-lm"])
        os.replace(tmp, _SO)
    return _SO


_lib = None


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_SO)
        lib.syn_make_table.restype = ctypes.c_int
        lib.syn_make_table.argtypes = [ctypes.POINTER(_TableSpec), ctypes.POINTER(_ColSpec),
                                       ctypes.POINTER(_Col), ctypes.c_int64, ctypes.POINTER(_Col)]
        lib.syn_free_cols.restype = None
        lib.syn_free_cols.argtypes = [ctypes.POINTER(_Col), ctypes.c_int32]
        lib.syn_mix.restype = ctypes.c_uint64
        lib.syn_mix.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
        _lib = lib
    return _lib


@dataclass
class Column:
    name: str
    type: str                      # "string" | "int32" | "fp32"
    data: np.ndarray
    offsets: np.ndarray | None = None
    valid: np.ndarray | None = None

    def value(self, i: int):
        """Python value of row i (None when missing); for tests and fixtures."""
        if self.valid is not None and not self.valid[i]:
            return None
        if self.type == "string":
            return bytes(self.data[self.offsets[i]:self.offsets[i + 1]])
        return self.data[i].item()


@dataclass
class Table:
    columns: list[Column]
    n_rows: int
    job_offsets: np.ndarray | None = None    # int64[n_jobs+1] row ranges of independent jobs
    meta: dict = field(default_factory=dict)

    def col(self, name: str) -> int:
        return [c.name for c in self.columns].index(name)

    def slice(self, lo: int, hi: int) -> "Table":
        cols = []
        for c in self.columns:
            v = None if c.valid is None else c.valid[lo:hi].copy()
            if c.type == "string":
                o = c.offsets[lo:hi + 1].astype(np.int64)
                cols.append(Column(c.name, c.type, c.data[o[0]:o[-1]].copy(), (o - o[0]).astype(np.uint32), v))
            else:
                cols.append(Column(c.name, c.type, c.data[lo:hi].copy(), None, v))
        return Table(cols, hi - lo)

    def take(self, rows: np.ndarray) -> "Table":
        """Rows in the given order (a sub-relation for sampled checks)."""
        rows = np.asarray(rows, dtype=np.int64)
        cols = []
        for c in self.columns:
            v = None if c.valid is None else c.valid[rows].copy()
            if c.type == "string":
                o = c.offsets.astype(np.int64)
                lens = o[rows + 1] - o[rows]
                off = np.zeros(len(rows) + 1, np.int64)
                np.cumsum(lens, out=off[1:])
                idx = np.repeat(o[rows] - off[:-1], lens) + np.arange(off[-1])
                cols.append(Column(c.name, c.type, c.data[idx].copy(), off.astype(np.uint32), v))
            else:
                cols.append(Column(c.name, c.type, c.data[rows].copy(), None, v))
        return Table(cols, len(rows))

    def nbytes(self) -> int:
        t = 0
        for c in self.columns:
            t += c.data.nbytes + (0 if c.offsets is None else c.offsets.nbytes) + \
                (0 if c.valid is None else c.valid.nbytes)
        return t


def _spec(kind, lo=0, hi=0, card=0, s=1.1, mu=3.0, sigma=1.0, null_rate=0.0, edit=1):
    return (kind, lo, hi, card, s, mu, sigma, null_rate, edit)


def make_table(names, specs, n_rows, seed, dup_rate=0.0, cross_rate=0.0, edit_lo=1, edit_hi=3,
               swap_p=0.0, noise_rel=0.0, src: Table | None = None, shuffle=True) -> Table:
    lib = _load()
    nc = len(specs)
    cs = (_ColSpec * nc)()
    for i, sp in enumerate(specs):
        cs[i] = _ColSpec(sp[0], sp[1], sp[2], sp[3], sp[4], sp[5], sp[6], sp[7], sp[8], 0)
    ts = _TableSpec(n_rows, dup_rate, cross_rate, edit_lo, edit_hi, swap_p, noise_rel, seed, nc,
                    1 if shuffle else 0)
    out = (_Col * nc)()
    src_arr = None
    n_src = 0
    keep = []
    if src is not None:
        src_arr = (_Col * nc)()
        n_src = src.n_rows
        for i, c in enumerate(src.columns):
            valid = c.valid if c.valid is not None else np.ones(src.n_rows, np.uint8)
            keep.append(valid)
            col = _Col()
            col.n = src.n_rows
            col.valid = valid.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))
            if c.type == "string":
                col.type = 0
                col.bytes = c.data.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))
                col.off = c.offsets.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32))
            elif c.type == "int32":
                col.type = 1
                col.i32 = c.data.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
            else:
                col.type = 2
                col.f32 = c.data.ctypes.data_as(ctypes.POINTER(ctypes.c_float))
            src_arr[i] = col
    rc = lib.syn_make_table(ctypes.byref(ts), cs, src_arr, n_src, out)
    if rc != 0:
        raise MemoryError("synthetic table generation ran out of memory")
    cols = []
    try:
        for i in range(nc):
            o = out[i]
            valid = np.ctypeslib.as_array(o.valid, shape=(n_rows,)).copy() if n_rows else np.zeros(0, np.uint8)
            if valid.all():
                valid = None
            if o.type == 0:
                off = np.ctypeslib.as_array(o.off, shape=(n_rows + 1,)).copy()
                data = (np.ctypeslib.as_array(o.bytes, shape=(o.nbytes,)).copy() if o.nbytes
                        else np.zeros(0, np.uint8))
                cols.append(Column(names[i], "string", data, off, valid))
            elif o.type == 1:
                data = np.ctypeslib.as_array(o.i32, shape=(n_rows,)).copy() if n_rows else np.zeros(0, np.int32)
                cols.append(Column(names[i], "int32", data, None, valid))
            else:
                data = np.ctypeslib.as_array(o.f32, shape=(n_rows,)).copy() if n_rows else np.zeros(0, np.float32)
                cols.append(Column(names[i], "fp32", data, None, valid))
    finally:
        lib.syn_free_cols(out, nc)
    return Table(cols, n_rows)


def concat(tables: list[Table]) -> Table:
    """Stack tables with one schema into one (job_offsets marks the parts)."""
    cols = []
    for ci, c0 in enumerate(tables[0].columns):
        parts = [t.columns[ci] for t in tables]
        anynull = any(p.valid is not None for p in parts)
        valid = (np.concatenate([p.valid if p.valid is not None else np.ones(len(p.data) if p.type != "string"
                                 else len(p.offsets) - 1, np.uint8) for p in parts]) if anynull else None)
        if c0.type == "string":
            data = np.concatenate([p.data for p in parts])
            lens = np.concatenate([np.diff(p.offsets.astype(np.int64)) for p in parts])
            off = np.zeros(len(lens) + 1, np.int64)
            np.cumsum(lens, out=off[1:])
            cols.append(Column(c0.name, "string", data, off.astype(np.uint32), valid))
        else:
            cols.append(Column(c0.name, c0.type, np.concatenate([p.data for p in parts]), None, valid))
    sizes = np.array([t.n_rows for t in tables], np.int64)
    jo = np.zeros(len(tables) + 1, np.int64)
    np.cumsum(sizes, out=jo[1:])
    return Table(cols, int(jo[-1]), jo)


# ---------------------------------------------------------------- predicates / rules
def eq(c, cs=None):
    return ("eq", c, c if cs is None else cs, 0, 0, 0, 0, 0.0)


def eq_prefix(c, k, cs=None):
    return ("eq_prefix", c, c if cs is None else cs, k, 0, 0, 0, 0.0)


def ed(c, k, cs=None):
    return ("ed", c, c if cs is None else cs, k, 0, 0, 0, 0.0)


def jac(c, num, den, q=3, cs=None):
    return ("jaccard", c, c if cs is None else cs, 0, q, num, den, 0.0)


def absdiff(c, delta, cs=None):
    return ("absdiff", c, c if cs is None else cs, 0, 0, 0, 0, float(delta))


def const_eq(c, value, side=0):
    """t.A = c (side 0: the pair's first tuple) or s.A = c (side 1: its second)."""
    return ("const_eq", c, c, 0, 0, 0, 0, 0.0, side, value)


def contain(c, num, den, q=3, side=0, cs=None):
    """q-gram containment: |G(t.A) n G(s.B)| >= num/den of |G(t.A)| (side 0) or of |G(s.B)| (side 1)."""
    return ("contain", c, c if cs is None else cs, 0, q, num, den, 0.0, side)


def tjac(c, num, den, cs=None):
    """Jaccard similarity of the word-token sets (maximal runs of non-space bytes) >= num/den."""
    return ("tjaccard", c, c if cs is None else cs, 0, 0, num, den, 0.0)


BASE_SEED = 20241004

# ---------------------------------------------------------------- workload configurations
C2_NAMES = ["s1", "s2", "k1", "k2", "k3", "x1", "x2", "id"]


def _c2_specs(card1=1000, card2=10000, card3=100000, lo=8, hi=60):
    return [_spec(WORDS, lo, hi), _spec(WORDS, lo, hi),
            _spec(ZIPF_INT, card=card1, edit=0), _spec(ZIPF_STR, card=card2, edit=0),
            _spec(ZIPF_INT, card=card3, edit=0),
            _spec(LOGNORMAL, mu=3.0, sigma=1.0), _spec(LOGNORMAL, mu=3.0, sigma=1.0),
            _spec(ROWID, edit=0)]


def c2_mds():
    """Four rules over the 8-attribute schema (columns by index in C2_NAMES)."""
    s1, s2, k1, k2, k3, x1, x2 = 0, 1, 2, 3, 4, 5, 6
    return [
        [eq(k1), eq(k2), ed(s1, 2)],
        [eq(k2), eq(k3), jac(s1, 4, 5), absdiff(x1, 0.5)],
        [eq(k1), eq(k3), absdiff(x2, 1.0), ed(s2, 3)],
        [eq(k1), eq(k2), eq(k3), jac(s2, 7, 10)],
    ]


def config1(seed=BASE_SEED + 1, n=2000):
    """2,000 tuples: name a-z len 5-30, zip int32 over 500 values, city over 50
    values, price lognormal; 15% near-duplicates by 1-3 character edits."""
    specs = [_spec(LETTERS, 5, 30), _spec(UNIFORM_INT, card=500, edit=0),
             _spec(UNIFORM_STR, card=50, edit=0), _spec(LOGNORMAL, mu=3.0, sigma=1.0)]
    t = make_table(["name", "zip", "city", "price"], specs, n, seed, dup_rate=0.15, noise_rel=0.0)
    mds = [[eq(1), ed(0, 2)], [eq(2), jac(0, 4, 5)]]
    return t, mds


def config2(seed=BASE_SEED + 2, n=1_000_000, cards=(1000, 10000, 100000)):
    """Single table, 8 attributes, Zipf(1.1) keys, 10% near-duplicates."""
    t = make_table(C2_NAMES, _c2_specs(*cards), n, seed, dup_rate=0.10, swap_p=0.3, noise_rel=0.01)
    return t, c2_mds()


def c3_mds():
    s1, s2, k1 = 0, 1, 2
    return c2_mds() + [[eq_prefix(s1, 2), jac(s1, 4, 5)], [eq_prefix(s2, 2), eq(k1), ed(s2, 2)]]


def config3(seed=BASE_SEED + 3, n_r=500_000, n_s=2_000_000, cards=(1000, 10000, 100000)):
    """R x S: R and S share the 8-attribute schema; 5% of S rows derive from R rows."""
    r = make_table(C2_NAMES, _c2_specs(*cards), n_r, seed, dup_rate=0.0, swap_p=0.3, noise_rel=0.01)
    s = make_table(C2_NAMES, _c2_specs(*cards), n_s, seed + 7919, dup_rate=0.0, cross_rate=0.05,
                   swap_p=0.3, noise_rel=0.01, src=r)
    return r, s, c3_mds()


def c4_job_sizes(n_jobs=10_000, seed=BASE_SEED + 1004, lo=50, hi=20000):
    sizes = []
    for j in range(n_jobs):
        u1 = (_load().syn_mix(seed, 2 * j) >> 11) * (1.0 / 9007199254740992.0)
        u2 = (_load().syn_mix(seed, 2 * j + 1) >> 11) * (1.0 / 9007199254740992.0)
        z = math.sqrt(-2.0 * math.log(max(u1, 1e-300))) * math.cos(2 * math.pi * u2)
        sizes.append(int(min(hi, max(lo, round(math.exp(math.log(1000.0) + 1.2 * z))))))
    return sizes


def config4(n_jobs=10_000, seed=BASE_SEED + 1000, sizes=None):
    """Independent jobs of lognormal size in [50, 20000] with the C2 schema and
    rules; categorical cardinalities scale with the job size (minimum 5)."""
    if sizes is None:
        sizes = c4_job_sizes(n_jobs)
    parts = []
    for j, nj in enumerate(sizes):
        cards = tuple(max(5, int(round(c * nj / 1_000_000))) for c in (1000, 10000, 100000))
        parts.append(make_table(C2_NAMES, _c2_specs(*cards), nj, seed + j, dup_rate=0.10, swap_p=0.3,
                                noise_rel=0.01))
    t = concat(parts)
    return t, c2_mds()


C5_NAMES = ["s1", "s2", "s3", "s4", "c1", "c2", "c3", "c4", "c5", "x1", "x2", "x3"]


def c5_mds(seed=BASE_SEED + 5):
    """16 rules of 4-6 predicates: equality on 3 of the 5 categoricals, one or
    two string similarities (ED <= 2..3, or 3-gram Jaccard >= 7/10 or 4/5) and,
    for about half of them, |x - x'| <= delta on a numeric column."""
    lib = _load()
    mds = []
    for m in range(16):
        r = lambda k: lib.syn_mix(seed, m * 64 + k)
        cats = [4, 5, 6, 7, 8]
        chosen = []
        for k in range(3):
            chosen.append(cats.pop(int(r(k) % len(cats))))
        preds = [eq(c) for c in sorted(chosen)]
        strs = [0, 1, 2, 3]
        for j in range(1 + int(r(25) % 2)):       # one or two string similarities
            s = strs.pop(int(r(30 + j) % len(strs)))
            if r(20 + j) % 2 == 0:
                preds.append(ed(s, 2 + int(r(40 + j) % 2)))
            else:
                num, den = ((7, 10), (4, 5))[int(r(40 + j) % 2)]
                preds.append(jac(s, num, den))
        if r(50) % 2 == 0:
            preds.append(absdiff(9 + int(r(60) % 3), (0.5, 1.0, 2.0)[int(r(70) % 3)]))
        mds.append(preds)
    return mds


def config5(seed=BASE_SEED + 5, n=10_000_000):
    """10M tuples, 12 attributes: 4 strings (8-80), 5 Zipf(1.1) categoricals over
    1e3, 1e4, 1e4, 1e5, 1e5 values, 3 fp32 numerics; 10% near-duplicates."""
    specs = [_spec(WORDS, 8, 80) for _ in range(4)] + [
        _spec(ZIPF_INT, card=1000, edit=0), _spec(ZIPF_STR, card=10000, edit=0),
        _spec(ZIPF_INT, card=10000, edit=0), _spec(ZIPF_STR, card=100000, edit=0),
        _spec(ZIPF_INT, card=100000, edit=0)] + [_spec(LOGNORMAL, mu=3.0, sigma=1.0) for _ in range(3)]
    t = make_table(C5_NAMES, specs, n, seed, dup_rate=0.10, swap_p=0.3, noise_rel=0.01)
    return t, c5_mds()


def random_small(seed, n=300, null_rate=0.0, alphabet_small=False):
    """A small table with every column kind, optional missing values; used for
    edge-case parity (ties, nulls, empty strings, tiny blocks)."""
    lo, hi = (0, 12) if alphabet_small else (0, 40)
    specs = [_spec(LETTERS, lo, hi, null_rate=null_rate), _spec(WORDS, 3, 50, null_rate=null_rate),
             _spec(UNIFORM_INT, card=7, edit=0, null_rate=null_rate),
             _spec(ZIPF_STR, card=20, edit=0, null_rate=null_rate),
             _spec(LOGNORMAL, mu=1.0, sigma=0.5, null_rate=null_rate)]
    return make_table(["a", "b", "k", "c", "x"], specs, n, seed, dup_rate=0.3, swap_p=0.3, noise_rel=0.02)


def table_from_rows(names, types, rows) -> Table:
    """Build a Table from Python rows (None = missing); for hand-written fixtures."""
    n = len(rows)
    cols = []
    for ci, (name, ty) in enumerate(zip(names, types)):
        vals = [r[ci] for r in rows]
        valid = np.array([v is not None for v in vals], np.uint8)
        if ty == "string":
            bs = [(v.encode() if isinstance(v, str) else (v or b"")) for v in vals]
            off = np.zeros(n + 1, np.int64)
            np.cumsum([len(b) for b in bs], out=off[1:])
            data = np.frombuffer(b"".join(bs), np.uint8).copy() if off[-1] else np.zeros(0, np.uint8)
            cols.append(Column(name, ty, data, off.astype(np.uint32), None if valid.all() else valid))
        elif ty == "int32":
            cols.append(Column(name, ty, np.array([v or 0 for v in vals], np.int32), None,
                               None if valid.all() else valid))
        else:
            cols.append(Column(name, ty, np.array([v if v is not None else 0.0 for v in vals], np.float32),
                               None, None if valid.all() else valid))
    return Table(cols, n)


def random_rule_set(seed, n_mds, key_cols, str_cols, num_cols, n_keys=(2, 3)):
    """A seeded random set of MDs: each MD holds equality on n_keys of the
    key columns, one string similarity (edit distance or 3-gram Jaccard) and
    often |a-b| <= delta on a numeric column or a second edit distance."""
    lib = _load()
    mds = []
    for m in range(n_mds):
        r = lambda k: lib.syn_mix(seed, m * 97 + k)
        keys = list(key_cols)
        nk = n_keys[0] + int(r(0) % (n_keys[1] - n_keys[0] + 1))
        chosen = []
        for k in range(min(nk, len(keys))):
            chosen.append(keys.pop(int(r(1 + k) % len(keys))))
        preds = [eq(c) for c in sorted(chosen)]
        col = str_cols[int(r(30) % len(str_cols))]
        if r(20) % 2 == 0:
            preds.append(ed(col, 1 + int(r(40) % 3)))
        else:
            num, den = ((1, 2), (3, 5), (7, 10), (4, 5), (9, 10))[int(r(40) % 5)]
            preds.append(jac(col, num, den))
        if r(50) % 3 != 0:
            preds.append(absdiff(num_cols[int(r(60) % len(num_cols))], (0.1, 0.5, 1.0, 2.0, 5.0)[int(r(70) % 5)]))
        if r(80) % 2 == 0:
            other = [c for c in str_cols if c != col] or str_cols
            oc = other[int(r(90) % len(other))]
            if r(85) % 2 == 0:
                preds.append(ed(oc, 1 + int(r(95) % 3)))
            else:
                num, den = ((1, 2), (3, 5), (7, 10), (4, 5), (9, 10))[int(r(95) % 5)]
                preds.append(jac(oc, num, den))
        mds.append(preds)
    return mds
