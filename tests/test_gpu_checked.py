"""The GPU parity suites run again on the bounds-checked build
(libhb_checked.so, HB_CHECKED=1): every staged index of the evaluation
kernel and every output position of the encoder and block builder is checked
against its buffer there, and a failed check would turn the call into
HB_ERR_BOUNDS.  The suites must pass unchanged."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SUITES = ["tests/test_gpu_parity.py", "tests/test_gpu_general.py", "tests/test_gpu_partition.py",
          "tests/test_gpu_stream.py", "tests/test_gpu_batch.py", "tests/test_gpu_allpairs.py",
          "tests/test_gpu_errors.py"]


def _env():
    return dict(os.environ, HB_CHECKED="1")


def test_checked_library_is_the_one_loaded():
    r = subprocess.run([sys.executable, "-c", "from paper_2410_04349_gb300 import hb; "
                        "print(hb.lib().hb_version().decode())"], env=_env(), cwd=ROOT, capture_output=True,
                       text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    assert "checked" in r.stdout


def test_parity_suites_under_bounds_checks():
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", "-m", "gpu and not slow"]
                       + SUITES, env=_env(), cwd=ROOT, capture_output=True, text=True, timeout=3000)
    assert r.returncode == 0, r.stdout[-4000:] + r.stderr[-2000:]
