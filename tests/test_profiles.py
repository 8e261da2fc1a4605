"""The committed ncu summaries parse, and bench.py reads the DRAM traffic of the
evaluation kernel from them when the kernel source is the one profiled."""
import hashlib
import os

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _fields(path):
    text = open(path).read()
    return dict(line.split(": ", 1) for line in text.splitlines() if ": " in line)


def test_eval_kernel_summary_has_the_fields_bench_reads():
    f = _fields(os.path.join(ROOT, "profiles", "k_eval_c2.txt"))
    assert f["command"].startswith("ncu ") and "--clock-control none" in f["command"]
    assert len(f["k_eval.cu sha256[:16]"].strip()) == 16
    assert float(f["dram bytes per full launch"]) > 0


def test_bench_traffic_follows_the_kernel_source():
    f = _fields(os.path.join(ROOT, "profiles", "k_eval_c2.txt"))
    src = os.path.join(ROOT, "paper_2410_04349_gb300", "csrc", "k_eval.cu")
    sha = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    got = bench.eval_kernel_traffic()
    if f["k_eval.cu sha256[:16]"].strip() == sha:
        assert got == float(f["dram bytes per full launch"])
    else:
        assert got is None


def test_launch_list_names_its_command():
    text = open(os.path.join(ROOT, "profiles", "launches_c2.txt")).read()
    assert "ncu --metrics gpu__time_duration.sum --clock-control none" in text
    assert "k_eval" in text
