"""Host check of the periodic index wraps of the step kernels (no GPU).

wrap_near (the tile kernels' compare-and-add wrap with an integer-modulo
fallback) must equal the mathematical v mod n for every v and n; it is
compiled here from csrc/step_kernel.cuh by nvcc as host code and run over
n = 1..70 and v = -300..300.
"""
import os
import shutil
import subprocess

import pytest

CSRC = os.path.join(os.path.dirname(__file__), "..", "paper_0710_5470_gb300", "csrc")

PROG = r"""
#include <cstdio>
#include "step_kernel.cuh"
int main() {
    for (int n = 1; n <= 70; ++n)
        for (int v = -300; v <= 300; ++v)
            std::printf("%d %d %d %d\n", n, v, lbk::wrap_near(v, n), lbk::wrapi(v, n));
    return 0;
}
"""


def test_wrap_near_is_modulo(tmp_path):
    from paper_0710_5470_gb300 import build
    nvcc = build.nvcc()
    if not shutil.which(nvcc) and not os.path.exists(nvcc):
        pytest.skip("nvcc not found")
    src = tmp_path / "wrap.cu"
    src.write_text(PROG)
    exe = tmp_path / "wrap"
    subprocess.run([nvcc] + build.ARCH + ["-std=c++17", "--expt-relaxed-constexpr", "-I", CSRC, "-I",
                    os.path.join(CSRC, "..", "..", "include"), str(src), "-o", str(exe)],
                   check=True, capture_output=True, text=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    count = 0
    for line in out:
        if not line:
            continue
        n, v, near, mod = map(int, line.split())
        assert near == v % n and mod == v % n, (n, v, near, mod)
        count += 1
    assert count == 70 * 601
