"""Host-side limits of the block build, checked without a GPU: the helper that
decides whether the member lists of all active MDs fit 32-bit addressing (used
by hb_block and by hb_block_stream before any device work) is compiled into a
small host program and probed at the boundary."""
import os
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2410_04349_gb300", "csrc")
CUDA_INC = "/usr/local/cuda/include"

PROBE = r"""
#include <cstdio>
#include "hb_internal.h"
int main() {
    long long cases[][2] = {{1, 4294967295LL}, {1, 4294967296LL}, {64, 67108863LL}, {64, 67108864LL},
                            {0, 4294967295LL}, {6, 0}, {4, 1073741824LL}, {3, 1431655765LL}, {3, 1431655766LL}};
    for (auto &c : cases) std::printf("%d\n", hb::member_addressing_fits(c[0], c[1]) ? 1 : 0);
    return 0;
}
"""


def test_member_addressing_boundary(tmp_path):
    if not os.path.isdir(CUDA_INC):
        pytest.skip("CUDA headers not installed")
    src = tmp_path / "probe.cpp"
    src.write_text(PROBE)
    exe = tmp_path / "probe"
    subprocess.check_call(["g++", "-std=c++17", "-I", CSRC, "-I", os.path.join(ROOT, "include"), "-I", CUDA_INC,
                           str(src), "-o", str(exe)])
    out = subprocess.check_output([str(exe)], text=True).split()
    # 2^32 - 1 members fit, 2^32 do not (64 MDs x 2^26 rows = 2^32)
    assert out == ["1", "0", "1", "0", "1", "1", "0", "1", "0"]
