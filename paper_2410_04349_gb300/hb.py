"""ctypes binding of libhb (include/hb.h): argument marshalling only.

Every step of blocking runs in the library's CUDA kernels; this module only
turns Python/numpy/torch objects into the C structs and pointers of the
C-ABI and back.  It raises if libhb.so has not been built: there is no
fallback implementation.

Columns are passed as objects with attributes ``type`` ("string", "int32",
"fp32"), ``data`` (numpy array or torch tensor), ``offsets`` (strings: n+1
uint32) and ``valid`` (uint8 per row or None).  Tensors on a CUDA device are
passed as device pointers (``on_device=True``).

Predicates are tuples ``(kind, col_t, col_s, k, q, num, den, delta[, side[, value]])``
with kind in {"eq", "eq_prefix", "ed", "jaccard", "absdiff", "const_eq", "contain",
"tjaccard"}; side and value carry a constant's side and bytes (or int) and a
containment's dividing side.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# HB_CHECKED=1 in the environment loads the bounds-checked build (libhb_checked.so)
LIB_PATH = os.path.join(_HERE, "libhb_checked.so" if os.environ.get("HB_CHECKED") == "1" else "libhb.so")

HB_OK, HB_ERR_ARG, HB_ERR_OOM, HB_ERR_CUDA, HB_ERR_STATE, HB_ERR_OVERFLOW, HB_ERR_DEVICE_TIMEOUT = 0, -1, -2, -3, -4, -5, -6
KINDS = {"eq": 0, "eq_prefix": 1, "ed": 2, "jaccard": 3, "absdiff": 4, "const_eq": 5, "contain": 6, "tjaccard": 7}
TYPES = {"string": 0, "int32": 1, "fp32": 2}
FLAG_PER_JOB_LAUNCHES, FLAG_NO_GRAPH = 1, 2
PLAN_MODES = {"rule_data": 0, "learned": 1, "given": 2, "random": 3, "cost_first": 4, "sel_first": 5}
MAX_MDS, MAX_PREDS, FEATURES = 64, 128, 32
PAIR_FEATURES = 8
PAIR_MODEL_PARAMS = 8 * 2 + 2 + 2 * 6 + 6 + 6 + 1
MLP_PARAMS = 32 * 64 + 64 + 64 * 64 + 64 + 64 + 1


class HBError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"libhb status {status}: {msg}")
        self.status = status


class hb_column(ctypes.Structure):
    _fields_ = [("type", ctypes.c_int32), ("reserved", ctypes.c_int32), ("data", ctypes.c_void_p),
                ("offsets", ctypes.c_void_p), ("valid", ctypes.c_void_p), ("data_bytes", ctypes.c_uint64)]


class hb_predicate(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("col_t", ctypes.c_int32), ("col_s", ctypes.c_int32),
                ("k", ctypes.c_int32), ("q", ctypes.c_int32), ("num", ctypes.c_uint32), ("den", ctypes.c_uint32),
                ("delta", ctypes.c_float), ("side", ctypes.c_int32), ("value_len", ctypes.c_uint32),
                ("value", ctypes.c_void_p)]


class hb_pair(ctypes.Structure):
    _fields_ = [("tid1", ctypes.c_uint32), ("tid2", ctypes.c_uint32)]


class hb_options(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int32), ("tile", ctypes.c_int32), ("chunk_bytes", ctypes.c_uint64),
                ("seed", ctypes.c_uint64), ("stream", ctypes.c_void_p), ("out_capacity", ctypes.c_int64),
                ("flags", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class hb_plan_info(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int32), ("n_preds", ctypes.c_int32), ("n_ops", ctypes.c_int32),
                ("n_eq", ctypes.c_int32), ("op_pred", ctypes.c_int32 * MAX_PREDS),
                ("md_order", ctypes.c_int32 * MAX_MDS), ("sp", ctypes.c_double * MAX_PREDS),
                ("cost", ctypes.c_double * MAX_PREDS), ("pred_md", ctypes.c_int32 * MAX_PREDS),
                ("tile", ctypes.c_int32), ("n_mds", ctypes.c_int32), ("record_words", ctypes.c_int32),
                ("hot_words", ctypes.c_int32), ("n_branches", ctypes.c_int32),
                ("branch_pred", ctypes.c_int32 * MAX_MDS)]


class hb_stats(ctypes.Structure):
    _fields_ = [("n_rows_r", ctypes.c_int64), ("n_rows_s", ctypes.c_int64), ("candidate_pairs", ctypes.c_int64),
                ("emitted_pairs", ctypes.c_int64), ("tiles", ctypes.c_int64), ("blocks", ctypes.c_int64),
                ("ms_h2d", ctypes.c_double), ("ms_encode", ctypes.c_double), ("ms_plan", ctypes.c_double),
                ("ms_block_build", ctypes.c_double), ("ms_eval", ctypes.c_double), ("ms_sort", ctypes.c_double),
                ("ms_d2h", ctypes.c_double), ("ms_total", ctypes.c_double), ("device_bytes", ctypes.c_int64),
                ("tile", ctypes.c_int32), ("n_mds", ctypes.c_int32), ("kernel_launches", ctypes.c_int64),
                ("examined_pairs", ctypes.c_int64)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class hb_pred_log(ctypes.Structure):
    _fields_ = [("features", ctypes.c_float * FEATURES), ("log_cost", ctypes.c_float),
                ("logit_pass", ctypes.c_float), ("evaluated", ctypes.c_int64), ("passed", ctypes.c_int64),
                ("cycles", ctypes.c_int64), ("stage1", ctypes.c_int64), ("stage2", ctypes.c_int64),
                ("core", ctypes.c_int64), ("pred", ctypes.c_int32), ("kind", ctypes.c_int32)]

    def as_dict(self):
        d = {f: getattr(self, f) for f, _ in self._fields_ if f != "features"}
        d["features"] = list(self.features)
        return d


EXPORTS = ["hb_create", "hb_destroy", "hb_last_error", "hb_version", "hb_load_table", "hb_add_md", "hb_clear_mds",
           "hb_plan", "hb_block", "hb_block_device", "hb_block_stream", "hb_block_batch", "hb_free_pairs",
           "hb_get_stats", "hb_plan_order", "hb_log_predicates", "hb_predicate_features", "hb_train_cost_model",
           "hb_get_cost_model", "hb_set_cost_model", "hb_mlp_forward", "hb_mlp_forward_bf16", "hb_mlp_backward",
           "hb_mlp_backward_noalloc", "hb_adam_step", "hb_probe_int_issue", "hb_time_pairs",
           "hb_pair_model_forward", "hb_pair_model_backward", "hb_train_pair_model", "hb_tile_log",
           "hb_train_tile_model", "hb_set_tile_model", "hb_get_tile_model", "hb_batch_tile", "hb_set_partitions",
           "hb_set_shard", "hb_merge_pairs"]

_lib = None


def lib():
    """Load libhb.so; raises when it has not been built (no fallback exists)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2410_04349_gb300.build.build()")
    L = ctypes.CDLL(LIB_PATH)
    P, i32, i64, st = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_int
    sig = {
        "hb_create": (st, [P, P]), "hb_destroy": (None, [P]), "hb_last_error": (ctypes.c_char_p, []),
        "hb_version": (ctypes.c_char_p, []), "hb_load_table": (st, [P, i32, i64, i32, P, i32]),
        "hb_add_md": (st, [P, i32, P, P]), "hb_clear_mds": (st, [P]), "hb_plan": (st, [P, i32, P]),
        "hb_block": (st, [P, P, P]), "hb_block_device": (st, [P, P, P]),
        "hb_block_stream": (st, [P, i64, i32, P, P, P]), "hb_block_batch": (st, [P, i32, P, P, P]),
        "hb_free_pairs": (None, [P]), "hb_get_stats": (st, [P, P]),
        "hb_plan_order": (st, [i32, P, P, i32, P, P, P, P, P, P, P]),
        "hb_log_predicates": (st, [P, i32, P, i32, P]), "hb_predicate_features": (st, [P, P, i32, P]),
        "hb_train_cost_model": (st, [P, i32, P, P, P, i32, ctypes.c_float, ctypes.c_uint64, P]),
        "hb_get_cost_model": (st, [P, P]), "hb_set_cost_model": (st, [P, P]),
        "hb_mlp_forward": (st, [P, i32, P, P, P]), "hb_mlp_forward_bf16": (st, [P, i32, P, P, P]),
        "hb_mlp_backward": (st, [P, P, i32, P, P, P]), "hb_mlp_backward_noalloc": (st, [P, P, i32, P, P, P]),
        "hb_adam_step": (st, [P, P, P, P, i32, i32, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                              P]),
        "hb_probe_int_issue": (st, [i32, P, P, P]),
        "hb_time_pairs": (st, [P, i32, i32, P, P, P, P, P]),
        "hb_pair_model_forward": (st, [P, i32, P, P, P]),
        "hb_pair_model_backward": (st, [P, P, i32, P, P, P]),
        "hb_train_pair_model": (st, [i32, P, P, i32, ctypes.c_float, ctypes.c_uint64, P, P]),
        "hb_tile_log": (st, [P, i32, P, P, P]),
        "hb_train_tile_model": (st, [P, i32, P, P, i32, ctypes.c_float, ctypes.c_uint64, P]),
        "hb_set_tile_model": (st, [P, P]), "hb_get_tile_model": (st, [P, P]),
        "hb_batch_tile": (st, [P, P, P, P]),
        "hb_set_partitions": (st, [P, ctypes.c_uint32]),
        "hb_set_shard": (st, [P, i32, i32]),
        "hb_merge_pairs": (st, [P, P, i32, P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def _check(status, what=""):
    if status != HB_OK:
        msg = lib().hb_last_error()
        raise HBError(status, f"{what}: {msg.decode() if msg else ''}")


def _ptr(x):
    """Raw address of a numpy array or torch tensor (None -> NULL)."""
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        return x.data_ptr() or None
    return x.ctypes.data if x.size else None


def _nbytes(x):
    if hasattr(x, "element_size"):
        return x.numel() * x.element_size()
    return x.nbytes


def _columns(cols):
    arr = (hb_column * max(len(cols), 1))()
    keep = []
    for i, c in enumerate(cols):
        data = c.data
        if not hasattr(data, "data_ptr"):
            data = np.ascontiguousarray(data)
        keep.append(data)
        hc = hb_column()
        hc.type = TYPES[c.type]
        hc.data = _ptr(data)
        if c.type == "string":
            off = c.offsets
            if not hasattr(off, "data_ptr"):
                off = np.ascontiguousarray(off, np.uint32)
            keep.append(off)
            hc.offsets = _ptr(off)
            hc.data_bytes = _nbytes(data)
        if c.valid is not None:
            v = c.valid
            if not hasattr(v, "data_ptr"):
                v = np.ascontiguousarray(v, np.uint8)
            keep.append(v)
            hc.valid = _ptr(v)
        arr[i] = hc
    return arr, keep


class PinnedColumn:
    """A column whose arrays live in page-locked host memory."""

    def __init__(self, col, keep):
        self.type = col.type
        self.data = _pin(col.data, keep)
        self.offsets = _pin(getattr(col, "offsets", None), keep)
        self.valid = _pin(getattr(col, "valid", None), keep)
        self._keep = keep


def _pin(a, keep):
    if a is None:
        return None
    import torch
    a = np.ascontiguousarray(a)
    t = torch.empty(max(a.nbytes, 1), dtype=torch.uint8, pin_memory=True)
    keep.append(t)
    v = t.numpy()[:a.nbytes].view(a.dtype).reshape(a.shape)
    v[...] = a
    return v


def pin_columns(columns):
    """Copies of host columns in page-locked memory (torch pin_memory): hb_load_table
    and hb_block_stream DMA such arrays directly instead of staging them."""
    return [PinnedColumn(c, []) for c in columns]


def _preds(md):
    """The C predicates of one MD; a constant's bytes (a string's, or an int32's
    little-endian 4) stay referenced by the returned array while hb_add_md
    copies them."""
    arr = (hb_predicate * len(md))()
    keep = []
    for i, p in enumerate(md):
        kind, ct, cs, k, q, num, den, delta = p[:8]
        side = p[8] if len(p) > 8 else 0
        arr[i] = hb_predicate(KINDS[kind], ct, cs, k, q, num, den, delta, side, 0, None)
        if kind == "const_eq":
            v = p[9]
            b = (v.encode() if isinstance(v, str) else bytes(v)) if isinstance(v, (str, bytes, bytearray)) \
                else np.array([v], np.int32).tobytes()
            buf = ctypes.create_string_buffer(b, max(len(b), 1))
            keep.append(buf)
            arr[i].value = ctypes.cast(buf, ctypes.c_void_p)
            arr[i].value_len = len(b)
    arr._keep = keep
    return arr


def _pairs_to_numpy(ptr, n):
    if n == 0:
        return np.zeros((0, 2), np.int64)
    buf = np.ctypeslib.as_array(ctypes.cast(ptr, ctypes.POINTER(ctypes.c_uint32)), shape=(n * 2,))
    return buf.reshape(n, 2).astype(np.int64)


class Context:
    """One libhb context (hb_create ... hb_destroy)."""

    def __init__(self, device=0, tile=0, chunk_bytes=0, seed=0, stream=None, out_capacity=0, flags=0):
        L = lib()
        opt = hb_options(device, tile, chunk_bytes, seed, stream, out_capacity, flags, 0)
        h = ctypes.c_void_p()
        _check(L.hb_create(ctypes.byref(h), ctypes.byref(opt)), "hb_create")
        self._h = h
        self._keep = []

    def close(self):
        if self._h:
            lib().hb_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # ---- tables and rules
    def load_table(self, side, n_rows, columns, on_device=False):
        arr, keep = _columns(columns)
        _check(lib().hb_load_table(self._h, side, n_rows, len(columns), arr, 1 if on_device else 0),
               "hb_load_table")

    def add_md(self, preds):
        out = ctypes.c_int32()
        _check(lib().hb_add_md(self._h, len(preds), _preds(preds), ctypes.byref(out)), "hb_add_md")
        return out.value

    def clear_mds(self):
        _check(lib().hb_clear_mds(self._h), "hb_clear_mds")

    def plan(self, mode="rule_data"):
        info = hb_plan_info()
        _check(lib().hb_plan(self._h, PLAN_MODES[mode] if isinstance(mode, str) else mode, ctypes.byref(info)),
               "hb_plan")
        return info

    def set_shard(self, rank, world):
        """Sharded evaluation: later blocking calls return the pairs of the
        blocks owned by `rank` of `world` (a function of each block's MD and
        smallest row); world = 1 evaluates everything."""
        _check(lib().hb_set_shard(self._h, int(rank), int(world)), "hb_set_shard")

    def set_partitions(self, m):
        """Root-edge hash partitioning (Section 5.3) with m partitions per hash
        function; 0 restores exact equality groups.  Applies from the next plan."""
        _check(lib().hb_set_partitions(self._h, int(m)), "hb_set_partitions")

    # ---- blocking
    def block(self):
        """Sorted unique pairs as int64 array [n, 2] (host)."""
        p = ctypes.c_void_p()
        n = ctypes.c_int64()
        _check(lib().hb_block(self._h, ctypes.byref(p), ctypes.byref(n)), "hb_block")
        try:
            return _pairs_to_numpy(p, n.value)
        finally:
            lib().hb_free_pairs(p)

    def block_device(self):
        """(device pointer of n sorted hb_pair, n); valid until the next call."""
        p = ctypes.c_void_p()
        n = ctypes.c_int64()
        _check(lib().hb_block_device(self._h, ctypes.byref(p), ctypes.byref(n)), "hb_block_device")
        return p.value, n.value

    def block_stream(self, n_rows_s, columns_s):
        arr, keep = _columns(columns_s)
        p = ctypes.c_void_p()
        n = ctypes.c_int64()
        _check(lib().hb_block_stream(self._h, n_rows_s, len(columns_s), arr, ctypes.byref(p), ctypes.byref(n)),
               "hb_block_stream")
        try:
            return _pairs_to_numpy(p, n.value)
        finally:
            lib().hb_free_pairs(p)

    def block_batch(self, job_rows):
        job_rows = np.ascontiguousarray(job_rows, np.int64)
        n_jobs = len(job_rows) - 1
        offs = np.zeros(n_jobs + 1, np.int64)
        p = ctypes.c_void_p()
        _check(lib().hb_block_batch(self._h, n_jobs, job_rows.ctypes.data, ctypes.byref(p), offs.ctypes.data),
               "hb_block_batch")
        try:
            return _pairs_to_numpy(p, int(offs[-1])), offs
        finally:
            lib().hb_free_pairs(p)

    def stats(self):
        s = hb_stats()
        _check(lib().hb_get_stats(self._h, ctypes.byref(s)), "hb_get_stats")
        return s.as_dict()

    # ---- learned cost model
    def log_predicates(self, profile=False, cap=MAX_PREDS):
        """Per-predicate instrumentation records (dicts) of one evaluation."""
        arr = (hb_pred_log * cap)()
        n = ctypes.c_int32()
        _check(lib().hb_log_predicates(self._h, 1 if profile else 0, arr, cap, ctypes.byref(n)),
               "hb_log_predicates")
        return [arr[i].as_dict() for i in range(n.value)]

    def predicate_features(self, cap=MAX_PREDS):
        out = np.zeros((cap, FEATURES), np.float32)
        n = ctypes.c_int32()
        _check(lib().hb_predicate_features(self._h, out.ctypes.data, cap, ctypes.byref(n)), "hb_predicate_features")
        return out[:n.value]

    def train_cost_model(self, X, y_cost, y_sel, epochs=300, lr=3e-3, seed=0):
        X = np.ascontiguousarray(X, np.float32)
        y_cost = np.ascontiguousarray(y_cost, np.float32)
        y_sel = np.ascontiguousarray(y_sel, np.float32)
        loss = np.zeros(2, np.float32)
        _check(lib().hb_train_cost_model(self._h, len(X), X.ctypes.data, y_cost.ctypes.data, y_sel.ctypes.data,
                                         epochs, lr, seed, loss.ctypes.data), "hb_train_cost_model")
        return loss

    def time_pairs(self, pred, i, j):
        """(cycles [n], verdicts [n], features [n, 8]) of checking distinct
        predicate pred on the pairs (i[k], j[k])."""
        i = np.ascontiguousarray(i, np.uint32)
        j = np.ascontiguousarray(j, np.uint32)
        n = len(i)
        cyc = np.zeros(max(n, 1), np.uint32)
        ver = np.zeros(max(n, 1), np.uint8)
        X = np.zeros((max(n, 1), PAIR_FEATURES), np.float32)
        _check(lib().hb_time_pairs(self._h, pred, n, i.ctypes.data, j.ctypes.data, cyc.ctypes.data, ver.ctypes.data,
                                   X.ctypes.data), "hb_time_pairs")
        return cyc[:n], ver[:n], X[:n]

    def tile_log(self):
        """(features [n, 32], log ms [n]) of every tile shape the batch autotuner timed."""
        n = ctypes.c_int32()
        _check(lib().hb_tile_log(self._h, 0, None, None, ctypes.byref(n)), "hb_tile_log")
        X = np.zeros((max(n.value, 1), FEATURES), np.float32)
        y = np.zeros(max(n.value, 1), np.float32)
        _check(lib().hb_tile_log(self._h, n.value, X.ctypes.data, y.ctypes.data, ctypes.byref(n)), "hb_tile_log")
        return X[:n.value], y[:n.value]

    def train_tile_model(self, X, y, epochs=1500, lr=2e-3, seed=0):
        X = np.ascontiguousarray(X, np.float32)
        y = np.ascontiguousarray(y, np.float32)
        loss = ctypes.c_float()
        _check(lib().hb_train_tile_model(self._h, len(y), X.ctypes.data, y.ctypes.data, epochs, lr, seed,
                                         ctypes.byref(loss)), "hb_train_tile_model")
        return loss.value

    def set_tile_model(self, params):
        if params is None:
            _check(lib().hb_set_tile_model(self._h, None), "hb_set_tile_model")
            return
        p = np.ascontiguousarray(params, np.float32)
        _check(lib().hb_set_tile_model(self._h, p.ctypes.data), "hb_set_tile_model")

    def get_tile_model(self):
        out = np.zeros(MLP_PARAMS, np.float32)
        _check(lib().hb_get_tile_model(self._h, out.ctypes.data), "hb_get_tile_model")
        return out

    def batch_tile(self):
        """(tile side, tiles per claim, 1 when the tile model chose them) of the last batch."""
        t, c, l = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        _check(lib().hb_batch_tile(self._h, ctypes.byref(t), ctypes.byref(c), ctypes.byref(l)), "hb_batch_tile")
        return t.value, c.value, l.value

    def get_cost_model(self):
        out = np.zeros(2 * MLP_PARAMS, np.float32)
        _check(lib().hb_get_cost_model(self._h, out.ctypes.data), "hb_get_cost_model")
        return out

    def set_cost_model(self, params):
        params = np.ascontiguousarray(params, np.float32)
        _check(lib().hb_set_cost_model(self._h, params.ctypes.data), "hb_set_cost_model")


def merge_pairs(lists):
    """k-way merge of sorted (n, 2) uint32 pair arrays into one sorted array
    (host code of the library)."""
    arrs = [np.ascontiguousarray(a, dtype=np.uint32).reshape(-1, 2) for a in lists]
    k = len(arrs)
    counts = np.array([a.shape[0] for a in arrs], dtype=np.int64)
    ptrs = (ctypes.c_void_p * max(k, 1))(*[a.ctypes.data for a in arrs])
    out = np.empty((int(counts.sum()), 2), dtype=np.uint32)
    _check(lib().hb_merge_pairs(ptrs, counts.ctypes.data if k else None, k, out.ctypes.data if out.size else None),
           "hb_merge_pairs")
    return out.astype(np.int64)


def plan_order(sp, cost, mds, skip=None):
    """Host-only ordering (hb_plan_order): (program, cp per MD, MD order)."""
    sp = np.ascontiguousarray(sp, np.float64)
    cost = np.ascontiguousarray(cost, np.float64)
    starts = np.zeros(len(mds) + 1, np.int32)
    flat = []
    for m, md in enumerate(mds):
        flat.extend(md)
        starts[m + 1] = len(flat)
    flat = np.ascontiguousarray(flat if flat else [0], np.int32)
    sk = None if skip is None else np.ascontiguousarray(skip, np.uint8)
    prog = np.zeros(MAX_PREDS, np.int32)
    n_prog = ctypes.c_int32()
    cp = np.zeros(max(len(mds), 1), np.int32)
    order = np.zeros(max(len(mds), 1), np.int32)
    _check(lib().hb_plan_order(len(sp), sp.ctypes.data, cost.ctypes.data, len(mds), starts.ctypes.data,
                               flat.ctypes.data, None if sk is None else sk.ctypes.data, prog.ctypes.data,
                               ctypes.byref(n_prog), cp.ctypes.data, order.ctypes.data), "hb_plan_order")
    return prog[:n_prog.value].tolist(), cp[:len(mds)].tolist(), order[:len(mds)].tolist()


def mlp_forward(X, params, y, stream=None, bf16=False):
    f = lib().hb_mlp_forward_bf16 if bf16 else lib().hb_mlp_forward
    _check(f(_ptr(X), X.shape[0], _ptr(params), _ptr(y), stream), "hb_mlp_forward")


def mlp_backward(X, t, params, grad, stream=None):
    _check(lib().hb_mlp_backward(_ptr(X), _ptr(t), X.shape[0], _ptr(params), _ptr(grad), stream), "hb_mlp_backward")


def mlp_backward_noalloc(X, t, params, grad, stream=None):
    """hb_mlp_backward for callers that cannot allocate device memory: the
    work buffers are a fixed array inside the library (n <= 4096 rows);
    concurrent calls on one GPU race on it."""
    _check(lib().hb_mlp_backward_noalloc(_ptr(X), _ptr(t), X.shape[0], _ptr(params), _ptr(grad), stream),
           "hb_mlp_backward_noalloc")


def adam_step(params, grad, m, v, step, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
    _check(lib().hb_adam_step(_ptr(params), _ptr(grad), _ptr(m), _ptr(v), params.numel(), step, lr, beta1, beta2,
                              eps, stream), "hb_adam_step")


def probe_int_issue(iters=4096, stream=None):
    """(integer operations per second, launch ms) of the library's issue-rate
    probe on the current device."""
    ops = ctypes.c_double()
    ms = ctypes.c_double()
    _check(lib().hb_probe_int_issue(iters, ctypes.byref(ops), ctypes.byref(ms), stream), "hb_probe_int_issue")
    return ops.value, ms.value


def pair_model_forward(X, params, y, stream=None):
    """The paper's per-pair model N on device tensors X [n, 8], params [43], y [n]."""
    _check(lib().hb_pair_model_forward(_ptr(X), X.shape[0], _ptr(params), _ptr(y), stream), "hb_pair_model_forward")


def pair_model_backward(X, t, params, grad, stream=None):
    _check(lib().hb_pair_model_backward(_ptr(X), _ptr(t), X.shape[0], _ptr(params), _ptr(grad), stream),
           "hb_pair_model_backward")


def train_pair_model(X, y, epochs=2000, lr=1e-2, seed=0):
    """(parameters [43], final mean squared error) of N trained on the GPU."""
    X = np.ascontiguousarray(X, np.float32)
    y = np.ascontiguousarray(y, np.float32)
    params = np.zeros(PAIR_MODEL_PARAMS, np.float32)
    loss = ctypes.c_float()
    _check(lib().hb_train_pair_model(len(y), X.ctypes.data, y.ctypes.data, epochs, lr, seed, params.ctypes.data,
                                     ctypes.byref(loss)), "hb_train_pair_model")
    return params, loss.value
