"""Host-side checks of the tensor-core staging layout and instruction descriptors
(paper_1707_05141_gb300/csrc/tcgen05.cuh), compiled with nvcc as a host program: no GPU needed."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "..")

PROG = r'''
#include <cstdio>
#include <vector>
#include "tcgen05.cuh"
using namespace bsvd::tc;
int main() {
    // the Gram stage: 128 operand rows (64 hi + 64 lo) x 32 K values, LBO 128, SBO 1024, 16 KB
    std::vector<int> seen(16384, 0);
    int bad = 0;
    for (int row = 0; row < 128; ++row)
        for (int k = 0; k < 32; ++k) {
            const unsigned off = kmajor_offset(row, k, 128, 1024);
            if (off % 4 != 0 || off + 4 > 16384) { ++bad; continue; }
            seen[off / 4] += 1;
        }
    for (int i = 0; i < 4096; ++i) if (seen[i] != 1) ++bad;
    // a core matrix is 8 rows x 16 contiguous bytes; K-adjacent core matrices are LBO apart
    if (kmajor_offset(1, 0, 128, 1024) != 16 || kmajor_offset(0, 4, 128, 1024) != 128 ||
        kmajor_offset(8, 0, 128, 1024) != 1024 || kmajor_offset(0, 1, 128, 1024) != 4) ++bad;
    printf("%d %u %u\n", bad, idesc_tf32(128, 128), idesc_tf32(128, 64));
    return 0;
}
'''


def test_gram_stage_layout_and_instruction_descriptors(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    src = tmp_path / "layout.cu"
    src.write_text(PROG)
    exe = tmp_path / "layout"
    inc = os.path.join(ROOT, "paper_1707_05141_gb300", "csrc")
    r = subprocess.run([nvcc, "-std=c++17", "-I", inc, str(src), "-o", str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()
    bad, id128, id64 = int(out[0]), int(out[1]), int(out[2])
    assert bad == 0
    # kind::tf32 instruction descriptor: D = F32 (bits 4-5 = 1), A = B = TF32 (bits 7-9, 10-12 = 2),
    # both K-major (bits 15, 16 = 0), N / 8 at bit 17, M / 16 at bit 24
    for val, m, n in ((id128, 128, 128), (id64, 128, 64)):
        assert (val >> 4) & 3 == 1 and (val >> 7) & 7 == 2 and (val >> 10) & 7 == 2
        assert (val >> 13) & 0xF == 0                       # no negation, K-major A and B
        assert (val >> 17) & 0x3F == n // 8 and (val >> 24) & 0x1F == m // 16
        assert val & 0xF == 0 and (val >> 23) & 1 == 0 and (val >> 29) == 0
