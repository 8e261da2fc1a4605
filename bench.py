#!/usr/bin/env python
"""Benchmark of rule-based blocking on GB300.

Workload: one relation of 1,000,000 tuples with 8 attributes (two strings of
8-60 characters in words, three Zipf(1.1) categorical keys over 10^3 / 10^4 /
10^5 values, two fp32 lognormal numerics, a row id), 10% near-duplicates made
by byte edits and word swaps, and four MDs of 3-4 predicates (equality on two
or three keys plus edit distance, 3-gram Jaccard and |a-b| <= delta).  The
data is seeded and synthetic (the paper's datasets are not available).

One step is the whole blocking path on the GPU: load the raw columns (already
in device memory), plan, encode, build blocks, evaluate every candidate pair,
compact and sort the result.  The metric is candidate pairs evaluated per
second (pairs that agree on all equality keys of some MD, each counted once).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gpu|reference]

With N > 1 (torchrun, one process per GPU) every rank blocks its own table
(seed + rank): the work is independent per rank, so scaling is weak and no
collective touches the data path.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "tuple pairs evaluated/sec"
UNIT = "pairs/s"
WORKLOAD = ("single table, 1,000,000 tuples x 8 attributes (2 strings 8-60 chars, 3 Zipf(1.1) keys over "
            "1e3/1e4/1e5 values, 2 fp32), 10% near-duplicates, 4 MDs")

GOLDEN = os.path.join(ROOT, "tests", "golden")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["gpu", "reference"], default="gpu")
    ap.add_argument("--rows", type=int, default=1_000_000)
    ap.add_argument("--cpu-sample-rows", type=int, default=80_000)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the learned-vs-plain (10M tuples) and batched-vs-per-job (10,000 jobs) comparisons")
    ap.add_argument("--workload", choices=["c2", "c3", "c4", "c5"], default="c2",
                    help="c2 (default): the single-table step above; c3: R x S with S streamed from host in pinned "
                         "chunks; c4: 10,000 jobs batched vs one launch sequence per job; c5: learned vs rule- and "
                         "data-aware plan on 10M tuples")
    return ap.parse_args()


def dist_env():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), \
        int(os.environ.get("LOCAL_RANK", "0"))


def aggregate(units: float, seconds: float, world: int):
    """Whole-job units and the slowest rank's time (all_reduce SUM / MAX)."""
    if world <= 1:
        return units, seconds
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    u = torch.tensor([units], dtype=torch.float64, device=dev)
    s = torch.tensor([seconds], dtype=torch.float64, device=dev)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    dist.all_reduce(s, op=dist.ReduceOp.MAX)
    return float(u.item()), float(s.item())


class ClockSampler:
    """nvidia-smi clock / throttle samples while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = tempfile.mktemp(suffix=".csv")

    def __enter__(self):
        try:
            self.out = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.out,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        try:
            self.out.close()
        except Exception:
            pass

    def summary(self):
        sm, mx, reasons = [], [], set()
        try:
            for line in open(self.path):
                f = [x.strip() for x in line.split(",")]
                if len(f) < 9:
                    continue
                try:
                    sm.append(float(f[1]))
                    mx.append(float(f[2]))
                except ValueError:
                    continue
                for name, v in zip(["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"],
                                   f[5:9]):
                    if v.lower() == "active":
                        reasons.add(name)
        except OSError:
            pass
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


def eval_kernel_traffic():
    """DRAM bytes per full-workload launch of the evaluation kernel from the
    committed ncu summary, or None when the kernel changed since it was taken."""
    path = os.path.join(ROOT, "profiles", "k_eval_c2.txt")
    src = os.path.join(ROOT, "paper_2410_04349_gb300", "csrc", "k_eval.cu")
    try:
        text = open(path).read()
        sha = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    except OSError:
        return None
    vals = dict(line.split(": ", 1) for line in text.splitlines() if ": " in line)
    if vals.get("k_eval.cu sha256[:16]", "").strip() != sha:
        return None
    try:
        return float(vals["dram bytes per full launch"].strip())
    except (KeyError, ValueError):
        return None


def plan_units(info, n_md):
    """Algorithmic integer work of one evaluation launch under the plan in use:
    the oracle's exact plan-replay count over every candidate pair of the
    full-size relation, stored by tests/golden/make_plan_units.py (committed
    data; nothing of the oracle runs here).  None when it was counted for
    another plan."""
    try:
        d = json.load(open(os.path.join(GOLDEN, "plan_units_c2.json")))
    except (OSError, ValueError):
        return None
    program = [int(x) for x in info.op_pred[:info.n_ops]]
    if d.get("program_ids") != program:
        return None
    return d


def algorithmic_bytes(table, mds, stats, q=3):
    """HBM bytes the encoder, the block build and the sort must move at least
    (the output each stage produces from the data it reads):
      encode: every column a rule reads, plus the dictionary code of each
        equality key (4 B a row), the q-gram lists of the Jaccard columns
        (4 B a gram, |s| - q + 1 grams for a string of |s| bytes) and their
        offsets (4 B a row);
      block build: per MD that builds blocks, its key codes read (4 B a key a
        row) and one member id written (4 B a row);
      sort: one read and one write of each 8-byte pair key per 8-bit radix pass
        over the used key bits."""
    n = table.n_rows
    used = sorted({p[1] for md in mds for p in md})
    read = 0
    for ci in used:
        c = table.columns[ci]
        read += c.data.nbytes + (0 if c.offsets is None else c.offsets.nbytes) + (0 if c.valid is None else c.valid.nbytes)
    eq_keys = {(p[0], p[1], p[3] if p[0] == "eq_prefix" else 0) for md in mds for p in md if p[0] in ("eq", "eq_prefix")}
    jac_cols = {(p[1], p[4]) for md in mds for p in md if p[0] == "jaccard"}
    grams = 0
    for ci, qq in jac_cols:
        lens = np.diff(table.columns[ci].offsets.astype(np.int64))
        grams += int(np.maximum(lens - qq + 1, 0).sum())
    enc = read + 4 * n * len(eq_keys) + 4 * grams + 4 * (n + 1) * len(jac_cols)
    eqsets = [frozenset((p[0], p[1], p[3] if p[0] == "eq_prefix" else 0) for p in md if p[0] in ("eq", "eq_prefix"))
              for md in mds]
    active = [m for m, e in enumerate(eqsets) if not any(eqsets[j] <= e for j in range(m))]
    blk = sum(4 * n * len(eqsets[m]) + 4 * n for m in active)
    bits = 2 * max(1, int(n - 1).bit_length())
    srt = 2 * 8 * stats["emitted_pairs"] * ((bits + 7) // 8)
    return {"encode": enc, "block_build": blk, "sort": srt}


def device_columns(table, device):
    import torch

    class Col:
        pass

    cols = []
    for c in table.columns:
        d = Col()
        d.type = c.type
        d.data = torch.from_numpy(c.data).to(device)
        d.offsets = torch.from_numpy(c.offsets.view(np.int32)).to(device) if c.offsets is not None else None
        d.valid = torch.from_numpy(c.valid).to(device) if c.valid is not None else None
        cols.append(d)
    return cols


def cpu_oracle_rate(table, mds, rows: int):
    """The oracle as it stands (grouped evaluation, all host threads) on the
    first `rows` tuples: (pairs/s, seconds, candidate pairs, threads)."""
    import oracle
    sub = table.slice(0, min(rows, table.n_rows))
    threads = os.cpu_count() or 1
    t0 = time.perf_counter()
    _, cand = oracle.block_hash(sub, mds, threads=threads)
    dt = time.perf_counter() - t0
    return cand / dt, dt, cand, threads


def run_reference(args, rank, world):
    """The oracle on the host cores (this tier's reference arm)."""
    if rank != 0:
        return 0
    import synth
    t, mds = synth.config2(n=args.rows)
    rows = args.cpu_sample_rows // 2
    for _ in range(args.warmup):
        cpu_oracle_rate(t, mds, rows)
    rates, secs, cand, threads = [], [], 0, 1
    for _ in range(args.steps):
        r, dt, cand, threads = cpu_oracle_rate(t, mds, rows)
        rates.append(r)
        secs.append(dt)
    value = cand * len(secs) / sum(secs)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(secs) / len(secs),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample": f"first {rows} tuples", "l2": "n/a (CPU)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": f"grouped oracle on the first {rows} of {args.rows} tuples, {cand} candidate pairs"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def _line(metric, value, unit, args, ms, workload, **extra):
    d = {"metric": metric, "value": value, "unit": unit, "n_gpus": 1, "steps": args.steps,
         "warmup": max(args.warmup, 3), "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
         "vs_baseline": None, "dtype": "u32", "data": "synthetic", "config": {"workload": workload}}
    d.update(extra)
    return d


def run_c3(args):
    """R (500K) x S (2M), six MDs, S streamed from host in pinned chunks."""
    import torch
    import synth
    from paper_2410_04349_gb300 import hb
    r, s, mds = synth.config3()
    s_locked = hb.pin_columns(s.columns)   # S in page-locked host memory: chunks are DMA'd straight from it
    out = {}
    for key, chunk, cols in (("256", 256 << 20, s_locked), ("32", 32 << 20, s_locked),
                             ("256_pageable", 256 << 20, s.columns)):
        with hb.Context(device=0, chunk_bytes=chunk) as ctx:
            ctx.load_table(0, r.n_rows, r.columns)
            for md in mds:
                ctx.add_md(md)
            for _ in range(max(args.warmup, 3)):
                pairs = ctx.block_stream(s.n_rows, cols)
            times = []
            for _ in range(args.steps):
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                pairs = ctx.block_stream(s.n_rows, cols)
                times.append(time.perf_counter() - t0)
            st = ctx.stats()
        out[key] = (statistics.median(times), st, len(pairs))
    t, st, n = out["256"]
    line = _line(METRIC, st["candidate_pairs"] / t, UNIT, args, t * 1e3,
                 "R x S: 500,000 x 2,000,000 tuples x 8 attributes, 5% cross-duplicates, 6 MDs (one blocked only by a "
                 "2-character prefix); S streamed from page-locked host memory in 256 MiB chunks",
                 candidate_pairs_per_step=st["candidate_pairs"], emitted_pairs_per_step=n,
                 e2e={"value": st["candidate_pairs"] / t, "unit": UNIT, "h2d_bytes_per_step": s.nbytes(),
                      "d2h_bytes_per_step": n * 8},
                 chunk_32MiB={"ms_per_step": out["32"][0] * 1e3,
                              "value": out["32"][1]["candidate_pairs"] / out["32"][0]},
                 pageable_S_256MiB={"ms_per_step": out["256_pageable"][0] * 1e3,
                                    "value": out["256_pageable"][1]["candidate_pairs"] / out["256_pageable"][0]})
    print(json.dumps(line), flush=True)
    return 0


def compare_c4(args):
    """10,000 independent jobs: one batched launch sequence (replayed from a
    CUDA graph, autotuned tile shape) vs one launch sequence per job, with the
    pair sets compared."""
    import torch
    import synth
    from paper_2410_04349_gb300 import hb
    t, mds = synth.config4()
    res = {}
    first, shapes = {}, {}
    tile_model = np.load(os.path.join(ROOT, "paper_2410_04349_gb300", "tile_model.npy"))
    for name, flags, steps, tm in (("batched", 0, args.steps, None), ("learned_tile", 0, args.steps, tile_model),
                                   ("per_job", hb.FLAG_PER_JOB_LAUNCHES, 1, None)):
        with hb.Context(device=0, flags=flags) as ctx:
            ctx.load_table(0, t.n_rows, t.columns)
            for md in mds:
                ctx.add_md(md)
            if tm is not None:
                ctx.set_tile_model(tm)
            torch.cuda.synchronize()
            f0 = time.perf_counter()
            pairs, offs = ctx.block_batch(t.job_offsets)   # first call: tile shape chosen, graph captured
            first[name] = time.perf_counter() - f0
            if not flags:
                shapes[name] = ctx.batch_tile()
            for _ in range(0 if flags else max(args.warmup, 3) - 1):
                pairs, offs = ctx.block_batch(t.job_offsets)
            times = []
            l0 = ctx.stats()["kernel_launches"]
            for _ in range(steps):
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                pairs, offs = ctx.block_batch(t.job_offsets)
                times.append(time.perf_counter() - t0)
            st = ctx.stats()
            res[name] = (statistics.median(times), st, pairs, offs, (st["kernel_launches"] - l0) // steps)
    tb, stb, pb, ob, lb = res["batched"]
    tp, stp, pp, op_, lp = res["per_job"]
    tl, stl, pl, ol, ll = res["learned_tile"]
    identical = bool(np.array_equal(pb, pp) and np.array_equal(ob, op_) and np.array_equal(pb, pl)
                     and np.array_equal(ob, ol))
    return {"workload": f"10,000 independent jobs, {t.n_rows} tuples in all (lognormal sizes in [50, 20000]), "
                        "C2 schema and rules, host-resident tables",
            "candidate_pairs": stb["candidate_pairs"], "emitted_pairs": int(len(pb)),
            "batched": {"ms_per_step": tb * 1e3, "value": stb["candidate_pairs"] / tb, "gpu_launches": lb,
                        "tile": stb["tile"], "steps": args.steps},
            "per_job": {"ms_per_step": tp * 1e3, "value": stp["candidate_pairs"] / tp, "gpu_launches": lp, "steps": 1},
            "learned_tile": {"ms_per_step": tl * 1e3, "first_call_ms": first["learned_tile"] * 1e3,
                             "autotuned_first_call_ms": first["batched"] * 1e3,
                             "shape": {"tile": shapes["learned_tile"][0], "claim": shapes["learned_tile"][1],
                                       "from_model": shapes["learned_tile"][2]},
                             "autotuned_shape": {"tile": shapes["batched"][0], "claim": shapes["batched"][1]}},
            "speedup": tp / tb, "identical_pair_sets": identical, "unit": UNIT,
            "timing": "wall clock around each hb_block_batch call (host tables in, pairs out), median"}


def measure_all_pairs(args):
    """The all-pairs path: 200,000 tuples of the single-table schema and one MD
    without an equality predicate (|x1 - x1'| <= 0.02 and ED(s1) <= 3), so every
    one of the 2.0e10 pairs is a candidate, evaluated through the tile queue."""
    import statistics as st_
    import synth
    from paper_2410_04349_gb300 import hb
    n = 200_000
    t, _ = synth.config2(n=n)
    mds = [[synth.absdiff(5, 0.02), synth.ed(0, 3)]]
    with hb.Context(device=0) as ctx:
        ctx.load_table(0, t.n_rows, t.columns)
        for md in mds:
            ctx.add_md(md)
        ctx.plan("rule_data")
        for _ in range(max(args.warmup, 3)):
            pairs = ctx.block()
        ev = []
        for _ in range(args.steps):
            pairs = ctx.block()
            ev.append(ctx.stats()["ms_eval"])
        st = ctx.stats()
    ms = st_.median(ev)
    return {"workload": "200,000 tuples x 8 attributes, one MD without equality (|x1 - x1'| <= 0.02 and "
                        "ED(s1) <= 3): every pair a candidate",
            "candidate_pairs": st["candidate_pairs"], "emitted_pairs": int(len(pairs)), "eval_ms": ms,
            "value": st["candidate_pairs"] / (ms / 1e3), "unit": UNIT,
            "timing": "CUDA events around the evaluation kernel, median"}


def measure_sharded(args, table, mds, world=4):
    """Sharded evaluation (hb_set_shard) of the step's table and rules, the
    ranks run one after the other on this GPU as separate processes would on
    theirs: each rank's evaluation time and candidate share (how evenly the
    owner function spreads the work), and whether the merged shards
    (hb_merge_pairs) equal the unsharded result."""
    import statistics as st_
    from paper_2410_04349_gb300 import hb
    runs, parts, whole = [], [], None
    for rank in range(-1, world):
        with hb.Context(device=0) as ctx:
            ctx.load_table(0, table.n_rows, table.columns)
            for md in mds:
                ctx.add_md(md)
            if rank >= 0:
                ctx.set_shard(rank, world)
            ctx.plan("rule_data")
            pairs = ctx.block()
            ev = []
            for _ in range(max(1, min(args.steps, 3))):
                pairs = ctx.block()
                ev.append(ctx.stats()["ms_eval"])
            stt = ctx.stats()
        if rank < 0:
            whole = pairs
            whole_ms = st_.median(ev)
            whole_cand = stt["candidate_pairs"]
            continue
        parts.append(pairs)
        runs.append({"rank": rank, "eval_ms": st_.median(ev), "candidate_pairs": stt["candidate_pairs"],
                     "emitted_pairs": int(len(pairs))})
    merged = hb.merge_pairs(parts)
    cand = [r["candidate_pairs"] for r in runs]
    return {"workload": f"the step's table and rules ({table.n_rows} tuples, {len(mds)} MDs) in {world} shards, "
                        "the ranks run in turn on one GPU", "world": world, "unsharded_eval_ms": whole_ms,
            "runs": runs, "max_rank_eval_ms": max(r["eval_ms"] for r in runs),
            "candidate_share_max_over_mean": max(cand) / (sum(cand) / world),
            "candidates_add_up": sum(cand) == whole_cand,
            "merged_equals_unsharded": bool(np.array_equal(merged, whole)),
            "timing": "CUDA events around the evaluation kernel, median"}


def measure_partitions(args, table, mds):
    """Root-edge hash partitioning (Section 5.3) on the step's own table and
    rules: m partitions per root-edge hash function instead of exact equality
    groups (m = 0).  The pair sets must be equal; the candidate count and the
    evaluation time show what coarser units cost on one GPU."""
    import statistics as st_
    from paper_2410_04349_gb300 import hb
    runs = []
    exact = None
    for m in (0, 1 << 20, 1 << 12):
        with hb.Context(device=0) as ctx:
            ctx.load_table(0, table.n_rows, table.columns)
            for md in mds:
                ctx.add_md(md)
            ctx.set_partitions(m)
            info = ctx.plan("rule_data")
            for _ in range(2):
                pairs = ctx.block()
            ev = []
            for _ in range(max(1, min(args.steps, 3))):
                pairs = ctx.block()
                ev.append(ctx.stats()["ms_eval"])
            st = ctx.stats()
        if exact is None:
            exact = pairs
        ms = st_.median(ev)
        runs.append({"m": m, "branches": int(info.n_branches), "candidate_pairs": st["candidate_pairs"],
                     "eval_ms": ms, "value": st["candidate_pairs"] / (ms / 1e3),
                     "identical_pair_sets": bool(np.array_equal(pairs, exact))})
    return {"workload": f"the step's table and rules ({table.n_rows} tuples, {len(mds)} MDs); m = 0: exact "
                        "equality groups, else m partitions per root-edge hash function", "unit": UNIT,
            "runs": runs, "timing": "CUDA events around the evaluation kernel, median"}


def run_c4(args):
    d = compare_c4(args)
    line = _line(METRIC, d["batched"]["value"], UNIT, args, d["batched"]["ms_per_step"], d["workload"],
                 batched_vs_per_job=d, gpu_launches=d["batched"]["gpu_launches"])
    print(json.dumps(line), flush=True)
    return 0 if d["identical_pair_sets"] else 1


MODEL_PATH = os.path.join(ROOT, "paper_2410_04349_gb300", "cost_model.npy")


def cost_model():
    """The committed cost model (two 32-64-64-1 networks trained on the blocker's
    logs of the C2-C4 workloads by paper_2410_04349_gb300/train_cost_model.py)."""
    return np.load(MODEL_PATH).astype(np.float32)


def compare_c5(args):
    """Learned plan (the committed cost model) vs the rule- and data-aware plan
    on 10M tuples x 12 attributes with 16 MDs; identical pair sets required."""
    import torch
    import synth
    from paper_2410_04349_gb300 import hb
    model = cost_model()
    t, mds = synth.config5()
    res = {}
    with hb.Context(device=0) as ctx:
        ctx.load_table(0, t.n_rows, t.columns)
        for md in mds:
            ctx.add_md(md)
        ctx.set_cost_model(model)
        for mode in ("rule_data", "learned"):
            tp0 = time.perf_counter()
            info = ctx.plan(mode)
            plan_s = time.perf_counter() - tp0
            for _ in range(max(args.warmup, 3)):
                pairs = ctx.block()
            ev, tot = [], []
            for _ in range(args.steps):
                torch.cuda.synchronize()
                s0 = time.perf_counter()
                pairs = ctx.block()
                tot.append(time.perf_counter() - s0)
                ev.append(ctx.stats()["ms_eval"])
            st = ctx.stats()
            res[mode] = {"eval_ms": statistics.median(ev), "step_ms": 1e3 * statistics.median(tot),
                         "plan_ms": plan_s * 1e3, "plan_mode_applied": int(info.mode), "tile": int(info.tile),
                         "program": [int(x) for x in info.op_pred[:info.n_ops]], "pairs": pairs, "st": st}
    L, Rd = res["learned"], res["rule_data"]
    identical = bool(np.array_equal(L["pairs"], Rd["pairs"]))
    cand = L["st"]["candidate_pairs"]
    out = {"workload": "single table, 10,000,000 tuples x 12 attributes (4 strings 8-80 chars, 5 Zipf(1.1) keys, "
                       "3 fp32), 10% near-duplicates, 16 MDs",
           "candidate_pairs": cand, "emitted_pairs": int(len(L["pairs"])), "unit": UNIT,
           "identical_pair_sets": identical,
           "eval_speedup_learned_vs_plain": Rd["eval_ms"] / L["eval_ms"],
           "step_speedup_learned_vs_plain": Rd["step_ms"] / L["step_ms"],
           "model": "paper_2410_04349_gb300/cost_model.npy",
           "timing": "eval_ms: CUDA events around the evaluation kernel; step_ms: wall clock around hb_block "
                     "(host tables already loaded), medians"}
    for k, v in (("learned", L), ("rule_data", Rd)):
        out[k] = {x: v[x] for x in ("eval_ms", "step_ms", "plan_ms", "plan_mode_applied", "tile", "program")}
        out[k]["value"] = cand / (v["eval_ms"] / 1e3)
    return out


def run_c5(args):
    d = compare_c5(args)
    line = _line(METRIC, d["learned"]["value"], UNIT, args, d["learned"]["step_ms"], d["workload"],
                 learned_vs_plain=d)
    print(json.dumps(line), flush=True)
    return 0 if d["identical_pair_sets"] else 1


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.workload != "c2":
        if rank != 0:
            return 0
        return {"c3": run_c3, "c4": run_c4, "c5": run_c5}[args.workload](args)
    import torch
    import synth
    from paper_2410_04349_gb300 import hb

    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    device = torch.device("cuda", local)
    torch.cuda.set_device(device)
    seed_offset = 1000 * rank   # every rank blocks its own seeded table (independent problems)
    table, mds = synth.config2(seed=synth.BASE_SEED + 2 + seed_offset, n=args.rows)
    dev_cols = device_columns(table, device)
    stream = torch.cuda.current_stream(device)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=device)
    ctx = hb.Context(device=local, stream=stream.cuda_stream)
    for md in mds:
        ctx.add_md(md)

    def step():
        ctx.load_table(0, table.n_rows, dev_cols, on_device=True)
        ctx.plan("rule_data")
        _, n_out = ctx.block_device()
        return n_out

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    # the integer issue-rate ceiling of this GPU, measured by the library's probe
    probe_ops, _ = hb.probe_int_issue(stream=stream.cuda_stream)
    probe_mhz = None
    torch.cuda.synchronize()
    launches0 = ctx.stats()["kernel_launches"]
    if world > 1:
        torch.distributed.barrier()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    eval_ms, cands, outs = [], [], []
    stage_hist = {"ms_encode": [], "ms_block_build": [], "ms_sort": []}
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        for i in range(args.steps):
            flush.zero_()                       # evict L2 (256 MiB > 129 MB) between steps
            ev[i][0].record(stream)
            n_out = step()
            ev[i][1].record(stream)
            st = ctx.stats()
            eval_ms.append(st["ms_eval"])
            for k in stage_hist:
                stage_hist[k].append(st[k])
            cands.append(st["candidate_pairs"])
            outs.append(n_out)
        torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    launches = ctx.stats()["kernel_launches"] - launches0
    step_ms = [a.elapsed_time(b) for a, b in ev]
    local_s = sum(step_ms) / 1e3
    units, secs = aggregate(float(sum(cands)), local_s, world)
    value = units / secs
    st = ctx.stats()

    # roofline of the evaluation kernel: algorithmic integer operations per
    # launch (the oracle's plan-replay count for the plan in use) over the
    # library's measured integer issue rate; its staged bytes against HBM
    info = ctx.plan("rule_data")
    clocks = clk.summary()
    sm_mhz = clocks["sm_mhz"] or measured_peaks().get("clocks_under_load", {}).get("sm_mhz_median", 1440.0)
    n_sm = torch.cuda.get_device_properties(device).multi_processor_count
    derived_ops = n_sm * 4 * 32 * sm_mhz * 1e6      # one 32-lane warp instruction per SMSP per clock
    eval_s = statistics.median(eval_ms) / 1e3
    pu = plan_units(info, len(mds)) if args.rows == 1_000_000 and seed_offset == 0 else None
    hbm = measured_peaks().get("hbm_gbs", 6800.0) * 1e9
    hw_bytes = 4 * info.hot_words
    staged = float(st["tiles"]) * 2 * (32 * info.tile // 32) * hw_bytes + 8.0 * outs[-1]
    roofline = {"bound": "alu", "kernel": "k_eval", "unit": "Tops/s", "launch_ms": eval_s * 1e3,
                "peak": probe_ops / 1e12,
                "peak_basis": f"measured by hb_probe_int_issue (8 independent add/shift/logic chains per thread, "
                              f"8 x 256-thread blocks per SM): {probe_ops / 1e12:.1f} T int ops/s at "
                              f"{probe_mhz or sm_mhz:.0f} MHz; derived {n_sm} SMs x 4 SMSPs x 32 lanes x clock = "
                              f"{derived_ops / 1e12:.1f} T",
                "traffic": eval_kernel_traffic(),
                "alg_bytes_per_launch": staged,
                "alg_bytes_basis": "hot records of both sides of every tile (tiles x 2 x 32 x hot-record bytes) "
                                   "+ 8 B per emitted pair",
                "hbm_frac": (staged / hbm) / eval_s}
    if pu is not None:
        ops = float(pu["units"]["total"])
        roofline.update({"achieved": ops / eval_s / 1e12, "frac": ops / eval_s / probe_ops,
                         "ops_per_launch": ops, "ops_basis": "oracle plan replay over all "
                         f"{pu['units']['candidates']} candidate pairs (tests/golden/plan_units_c2.json): "
                         + ", ".join(f"{k} {pu['units'][k]:.3g}" for k in ("eq", "owner", "absdiff", "ed", "jaccard"))})
    else:
        roofline.update({"achieved": None, "frac": None, "ops_per_launch": None,
                         "ops_basis": "no plan-replay count for this plan or size"})
    alg = algorithmic_bytes(table, mds, st)
    stage_ms = {k: st[k] for k in ("ms_encode", "ms_plan", "ms_block_build", "ms_eval", "ms_sort", "ms_d2h")}
    stages = {}
    for name, key in (("encode", "ms_encode"), ("block_build", "ms_block_build"), ("sort", "ms_sort")):
        t_s = statistics.median(stage_hist[key]) / 1e3
        stages[name] = {"bound": "hbm", "alg_bytes": alg[name], "ms": t_s * 1e3,
                        "achieved_gbs": alg[name] / t_s / 1e9 if t_s > 0 else None,
                        "frac": (alg[name] / hbm) / t_s if t_s > 0 else None}
    stages["eval"] = {"bound": "alu", "ms": eval_s * 1e3, "frac": roofline["frac"]}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": max(args.warmup, 3), "ms_per_step": secs * 1e3 / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n_tuples": table.n_rows, "n_mds": len(mds), "parallelism": f"dp{world}",
                   "l2": "flushed (256 MiB write) before every timed step", "inputs": "raw columns resident in HBM"},
        "candidate_pairs_per_step": cands[-1], "emitted_pairs_per_step": outs[-1],
        "examined_pairs_per_step": st["examined_pairs"],
        "eval_kernel_pairs_per_s": cands[-1] / eval_s,
        "stage_ms": stage_ms,
        "stage_roofline": stages,
        "gpu_launches": launches,
        "clocks": {"sm_mhz": clocks["sm_mhz"], "sm_max_mhz": clocks["sm_max_mhz"], "reasons": clocks["reasons"]},
        "roofline": roofline,
    }

    if not args.no_e2e:
        # the caller's columns in page-locked host memory; every step copies them
        # in and reads the sorted pairs back, over as many steps as the device-timed loop
        host_cols = hb.pin_columns(table.columns)
        h2d = table.nbytes()
        times, last_n = [], 0
        for i in range(max(args.warmup, 3) + args.steps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ctx.load_table(0, table.n_rows, host_cols, on_device=False)
            ctx.plan("rule_data")
            pairs = ctx.block()
            dt = time.perf_counter() - t0
            last_n = len(pairs)
            if i >= max(args.warmup, 3):
                times.append(dt)
        e2e_units, e2e_s = aggregate(float(cands[-1]) * len(times), sum(times), world)
        line["e2e"] = {"value": e2e_units / e2e_s, "unit": UNIT, "h2d_bytes_per_step": h2d,
                       "d2h_bytes_per_step": last_n * 8, "ms_per_step": 1e3 * e2e_s / len(times),
                       "steps": len(times)}
    ctx.close()

    if rank == 0 and world == 1 and not args.no_extra:
        # the metric's other halves: learned vs plain plan (10M tuples) and the
        # batched form vs one launch sequence per job (10,000 jobs)
        line["learned_vs_plain"] = compare_c5(args)
        line["batched_vs_per_job"] = compare_c4(args)
        line["all_pairs"] = measure_all_pairs(args)
        line["partitions"] = measure_partitions(args, table, mds)
        line["sharded"] = measure_sharded(args, table, mds)
    if rank == 0 and world == 1 and not args.no_cpu:
        rate, dt, cand, threads = cpu_oracle_rate(table, mds, args.cpu_sample_rows)
        line["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": threads, "kind": "oracle",
                                "sample": f"grouped oracle on the first {args.cpu_sample_rows} of {table.n_rows} "
                                          f"tuples: {cand} candidate pairs in {dt:.1f} s"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
