"""Build libhb.so in-tree for sm_103a (nvcc, one -gencode, parallel objects)."""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libhb.so")
# checked variant: device-side bounds checks that record a site instead of touching memory out of range
BUILD_CHECKED = os.path.join(HERE, "_build_checked")
LIB_CHECKED = os.path.join(HERE, "libhb_checked.so")

SOURCES = ["hb_api.cu", "hb_learn.cu", "k_sort.cu", "k_encode.cu", "k_block.cu", "k_eval.cu", "k_stats.cu",
           "k_mlp.cu", "planner.cpp", "hb_batch.cu", "hb_stream.cu", "k_probe.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _flags(verbose_ptx: bool, checked: bool):
    f = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-fvisibility=hidden",
         "-I", INCLUDE, "-I", CSRC, "--expt-relaxed-constexpr"] + ARCH
    if checked:
        f += ["-DHB_CHECKED"]
    if verbose_ptx:
        f += ["-Xptxas", "-v"]
    return f


def _compile(src: str, verbose_ptx: bool, checked: bool) -> str:
    obj = os.path.join(BUILD_CHECKED if checked else BUILD, os.path.splitext(src)[0] + ".o")
    path = os.path.join(CSRC, src)
    deps = [path] + [os.path.join(CSRC, h) for h in os.listdir(CSRC) if h.endswith(".h")] + \
        [os.path.join(INCLUDE, "hb.h")]
    if os.path.exists(obj) and not verbose_ptx and all(os.path.getmtime(obj) >= os.path.getmtime(d) for d in deps):
        return obj
    cmd = [nvcc()] + _flags(verbose_ptx, checked) + ["-c", path, "-o", obj + ".tmp"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
    if verbose_ptx and r.stderr:
        sys.stderr.write(r.stderr)
    os.replace(obj + ".tmp", obj)
    return obj


def _link(objs, lib) -> str:
    if os.path.exists(lib) and all(os.path.getmtime(lib) >= os.path.getmtime(o) for o in objs):
        return lib
    tmp = lib + f".tmp{os.getpid()}"
    cmd = [nvcc()] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib)
    return lib


def build(verbose_ptx: bool = False, checked: bool = True) -> str:
    """libhb.so, and with checked=True also libhb_checked.so (compiled in the same pool)."""
    variants = [False, True] if checked else [False]
    os.makedirs(BUILD, exist_ok=True)
    if checked:
        os.makedirs(BUILD_CHECKED, exist_ok=True)
    jobs = [(src, v) for v in variants for src in SOURCES]
    with cf.ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 4)) as ex:
        objs = list(ex.map(lambda j: _compile(j[0], verbose_ptx and not j[1], j[1]), jobs))
    _link(objs[:len(SOURCES)], LIB)
    if checked:
        _link(objs[len(SOURCES):], LIB_CHECKED)
    return LIB


if __name__ == "__main__":
    print(build(verbose_ptx="-v" in sys.argv))
