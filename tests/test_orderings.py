"""The round-robin ordering of Section 5 as the shared and block tiers use it (csrc/common.cuh),
compiled with nvcc as a host program (no GPU): every step pairs disjoint positions and one sweep
of np - 1 steps meets every pair exactly once; an odd column count runs with a padding position."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "..")

PROG = r'''
#include <cstdio>
#include <vector>
#include "common.cuh"
int main() {
    int bad = 0, checked = 0;
    for (int np = 2; np <= 258; np += 2) {
        std::vector<int> met(np * np, 0);
        for (int step = 0; step < np - 1; ++step) {
            std::vector<int> used(np, 0);
            for (int k = 0; k < np / 2; ++k) {
                int p = -1, q = -1;
                bsvd::round_robin_pair(np, step, k, p, q);
                if (!(0 <= p && p < q && q < np)) { ++bad; continue; }
                used[p] += 1; used[q] += 1; met[p * np + q] += 1;
            }
            for (int i = 0; i < np; ++i) bad += used[i] != 1;
        }
        for (int p = 0; p < np; ++p)
            for (int q = p + 1; q < np; ++q) bad += met[p * np + q] != 1;
        ++checked;
    }
    printf("%d %d\n", bad, checked);
    return 0;
}
'''


def test_round_robin_meets_every_pair_once_per_sweep(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    src = tmp_path / "rr.cu"
    src.write_text(PROG)
    exe = tmp_path / "rr"
    inc = [os.path.join(ROOT, "paper_1707_05141_gb300", "csrc"), os.path.join(ROOT, "include")]
    r = subprocess.run([nvcc, "-std=c++17", "-I", inc[0], "-I", inc[1], str(src), "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    bad, checked = map(int, subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split())
    assert checked == 129 and bad == 0


def _odd_even_exchange_sweeps(ns, sweeps=2):
    """The slot exchange of the columns-in-registers shared tier (csrc/jacobi_rx.cu) and of the
    register tier, restated: slot s holds columns (L, R); even steps rotate every slot, odd steps all
    but the wrap slot ns - 1; after an even step every slot takes its right neighbour's R, after an
    odd step every slot takes its left neighbour's L, except that the wrap slot hands over its R and
    keeps its L as the new R.  Yields the pairs met in each sweep of 2 ns steps."""
    L = [2 * s for s in range(ns)]
    R = [2 * s + 1 for s in range(ns)]
    for _ in range(sweeps):
        met = []
        for st in range(2 * ns):
            odd = st & 1
            met += [frozenset((L[s], R[s])) for s in range(ns) if not (odd and s == ns - 1)]
            if not odd:
                R = [R[(s + 1) % ns] for s in range(ns)]
            else:
                sent = [R[s] if s == ns - 1 else L[s] for s in range(ns)]
                R = [L[s] if s == ns - 1 else R[s] for s in range(ns)]
                L = [sent[(s - 1) % ns] for s in range(ns)]
        yield met


@pytest.mark.parametrize("ns", list(range(1, 65)))
def test_odd_even_exchange_meets_every_pair_once_per_sweep(ns):
    every = {frozenset((i, j)) for i in range(2 * ns) for j in range(i + 1, 2 * ns)}
    for met in _odd_even_exchange_sweeps(ns):
        assert len(met) == len(set(met)) and set(met) == every
