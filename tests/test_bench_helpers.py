"""Host-side helpers of bench.py (CPU only): the nvidia-smi clock-sample parser that decides
whether a timed run saw throttling, and the algorithmic flop count behind the roofline line."""
import numpy as np
import pytest

import bench


class _FakeProc:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def _clocks(lines):
    c = bench.Clocks(0)
    c.proc = _FakeProc()
    c.lines = lines
    return c


def _row(sm, mx=2070, hw="Not Active", hwt="Not Active", swt="Not Active", cap="Not Active"):
    return f"0, {sm}, {mx}, 812.4, 0x0000000000000000, {hw}, {hwt}, {swt}, {cap}"


def test_clock_samples_inside_the_timed_window_only(monkeypatch):
    monkeypatch.setattr(bench.time, "sleep", lambda s: None)
    lines = [(9.0, _row(1000, hw="Active")),          # before the window: ignored
             (10.5, _row(2060)), (11.0, _row(2070)), (11.5, _row(2055, cap="Active")),
             (13.0, _row(900, hwt="Active"))]         # after the window (+0.1 s): ignored
    out = _clocks(lines).stop(10.0, 12.0)
    assert out["samples"] == 3 and out["sm_mhz"] == 2060 and out["sm_max_mhz"] == 2070
    assert out["reasons"] == ["sw_power_cap"]


def test_clock_throttle_reasons_are_reported(monkeypatch):
    monkeypatch.setattr(bench.time, "sleep", lambda s: None)
    lines = [(1.0, _row(1500, hw="Active")), (1.1, _row(1400, hwt="Active")), (1.2, _row(1450, swt="Active")),
             (1.3, "garbage line"), (1.4, "0, [N/A], 2070, 1.0, 0x0, Not Active, Not Active, Not Active, Not Active")]
    out = _clocks(lines).stop(0.5, 2.0)
    assert out["reasons"] == ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"]
    assert out["samples"] == 3 and out["sm_mhz"] == 1450


def test_clocks_without_samples_or_tool():
    assert bench.Clocks(0).stop(0.0, 1.0) is None            # nvidia-smi never started
    out = _clocks([]).stop(0.0, 1.0)
    assert out["sm_mhz"] is None and out["samples"] == 0


def test_jacobi_flops_counts_pairs_and_rotations():
    # 4 x 4, 2 sweeps, 3 rotations: 2 sweeps x 6 pairs x 6 m + 3 x 6 (m + n)
    assert bench.jacobi_flops(4, 4, [2], [3]) == 2 * 6 * 24 + 3 * 6 * 8
    # a capped run reports NOT_CONVERGED + sweeps; the sweeps still count
    assert bench.jacobi_flops(4, 4, [(1 << 20) + 2], [3]) == bench.jacobi_flops(4, 4, [2], [3])
    # wide matrices pair the columns of A^T: k = min(m, n) columns of max(m, n) rows
    assert bench.jacobi_flops(3, 5, [1], [0]) == 1 * 3 * 6 * 5
    # preconditioning adds the factorisation (4 n^3 / 3) and the back-transformation (2 n^3) per matrix
    pre = bench.jacobi_flops(4, 4, [2, 2], [3, 3], precond=True) - bench.jacobi_flops(4, 4, [2, 2], [3, 3])
    assert pre == pytest.approx(2 * (4 * 64 / 3 + 2 * 64))


def test_traffic_entries_name_current_kernel_digests():
    for key, val in bench.TRAFFIC.items():
        name, digest = key.split(":")
        assert len(digest) == 16 and val > 0
        assert bench.kernel_digest(f"{name}.cu") == digest, f"{key}: kernel changed since its ncu capture"


def test_max_over_ranks_single_rank_is_identity():
    assert bench.max_over_ranks(3.25, 1, None) == 3.25


def test_launch_counts_follow_the_host_drivers():
    # block tier, 512 columns of width 32: 16 blocks, 15 steps x (Gram, inner SVD, polish, update)
    # and the sweep-end kernel for each of 20 sweeps, plus setup and finalize
    assert bench.block_jacobi_launches(512, 32, 20) == 1 + 20 * (15 * 4 + 1) + 1
    # randomized SVD of blocks up to 256 x 256, 4 rounds: plan + scan, 15 per round (the shared
    # tier joins the register tier for the small SVD), fallback + arrays, the QR path (4), the
    # shared tier, the block tier over 256 columns (8 blocks, 7 steps) and the finish kernel
    # the block tier on R^T of a blocked QR: setup, 8 panels, 7 trailing updates, R^T, the block
    # Jacobi, the zero fill, 8 block-reflector applications
    # per round: arrays, sample, 8 QR bins of Y, power step (8 + GEMM + 8 + GEMM), projection (GEMM + 8),
    # 2 small-SVD bins, 2 shared-tier bins, 2 GEMMs, estimate; then the full-rank path and the block
    # tier
    assert bench.rsvd_launches(256, 256, 4) == (2 + 4 * (1 + 1 + 8 + (8 + 1 + 8 + 1) + (1 + 8) + 2 + 2 + 2 + 1) + 2
                                               + (8 + 2 + 1 + 2)  # full rank: 8 QR bins, 2 + 1 SVDs, GEMM, copy
                                               + (1 + 8 + 7 + 1 + (1 + 20 * (7 * 4 + 1) + 1) + 1 + 8) + 1)
    # blocks up to 64 x 64: no shared or block tier
    assert bench.rsvd_launches(64, 64, 4) == 2 + 4 * (1 + 1 + 2 + (2 + 1 + 2 + 1) + (1 + 2) + 2 + 2 + 1) + 2 + (2 + 2 + 2) + 1
