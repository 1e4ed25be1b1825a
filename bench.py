#!/usr/bin/env python
"""Benchmark of the batched QR / Jacobi SVD / randomized SVD path on one GB300 (or N, weak scaling).

Default workload ``svd64_qr128``: one step = batched Householder QR of 20000 FP32 128 x 32 matrices
+ batched one-sided Jacobi SVD (U, S, V) of 20000 FP32 64 x 64 matrices (A = U diag(sigma) V^T,
Haar U, V, sigma_i = exp(-i/8)).  Metric: SVDs per second, whole job; inputs resident in HBM
(656 MB, larger than the 129 MB L2) when the timed region starts.

Other workloads (``--workload``), each printing its own line:
  fp64_32      1000 FP64 32 x 32 Jacobi SVDs + QRs, sigma_i = 10^(-8 i/31); the 8 MB batch fits in
               L2, so L2 is flushed before every timed step (outside that step's own events)
  block512     500 FP32 512 x 512 block-Jacobi SVDs (GRAM, block width 32), sigma log-uniform
  rsvd_uneven  16384 uneven blocks (m, n in {64, 128, 256}), randomized SVD to 1e-5 with the
               generator's rank as hint, the whole call captured in a CUDA graph
  hmatrix_mlp  ~52000 kernel blocks exp(-|x-y|/0.1) (3D points, k-d tree, leaf 64): randomized
               SVD to 1e-5 with ranks predicted by the learned network vs the plain adaptive method

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--workload NAME]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

# ALU peaks the FP32 / FP64 rooflines divide by.  Measured at start-up by the library's FMA probe
# (bsvd_fma_probe: 16 independent FMA chains per thread, 8 CTAs of 256 threads per SM, timed with
# CUDA events, best of five); the nominal figures below are used only when the probe cannot run.
PEAKS = {
    "fp32": {"tflops": 152 * 128 * 2 * 2.070e9 / 1e12,
             "note": "nominal FP32 SIMT: 152 SMs x 128 lanes x 2 flops x 2.07 GHz (probe not run)"},
    "fp64": {"tflops": 1.25, "note": "nominal FP64: GB300 data sheet (probe not run)"},
}


def measure_alu_peaks(bs, dev, local_rank=0):
    """FP32 and FP64 FMA throughput of this GPU (TFLOP/s), with the SM clock sampled meanwhile."""
    import torch
    stream = torch.cuda.current_stream()
    nsm = torch.cuda.get_device_properties(dev).multi_processor_count
    blocks = nsm * 8
    for key, code, iters, dt in (("fp32", bs.F32, 20000, torch.float32), ("fp64", bs.F64, 400, torch.float64)):
        out = torch.empty(blocks * 256, device=dev, dtype=dt)
        flops = bs.fma_probe(code, blocks, iters, out, stream)        # warm-up
        torch.cuda.synchronize()
        clocks = Clocks(local_rank)
        clocks.start()
        best = float("inf")
        w0 = time.time()
        for _ in range(5):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            bs.fma_probe(code, blocks, iters, out, stream)
            e1.record(stream)
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1))
        ck = clocks.stop(w0, time.time())
        PEAKS[key] = {"tflops": flops / (best * 1e-3) / 1e12,
                      "note": f"measured: bsvd_fma_probe ({blocks} CTAs x 256 threads x {iters} x 16 FMAs, "
                              f"best of 5 = {best:.3f} ms)", "clocks": ck}
    return PEAKS


def measured_hbm_gbs() -> float:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"])
    except (OSError, ValueError, KeyError):
        return 6800.0


# DRAM bytes (read + write) per launch of a dominant kernel from one ncu capture, keyed by the
# digest of the kernel's sources at capture time: a changed kernel has no entry and reports null
# traffic, not stale counters.  profiles/ holds the capture summaries.
TRAFFIC = {
    # jacobi_reg_kernel tier 0xa01, 10 000 64x64 matrices: 164.61 MB read + 277.57 MB written, per
    # 20 000-matrix launch (profiles/jacobi_reg_qr_svd64_qr128.md)
    "jacobi_reg:657c5a9dca399a6b": 2 * (164.607744e6 + 277.571072e6),
    # qr_warp_kernel<float, 128, 1>, 10 000 128x32 matrices: 164.79 MB read + 146.25 MB written, per
    # 20 000-matrix launch (re-captured after the CTA QR kernel's load phase changed in the same file)
    "qr:228caeb56544bd00": 2 * (164.788992e6 + 146.252800e6),
}


def kernel_digest(*names: str) -> str:
    h = hashlib.sha256()
    for name in names + ("common.cuh",):
        with open(os.path.join(ROOT, "paper_1707_05141_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


# ----------------------------------------------------------------------------------------------
# clocks sampler (nvidia-smi during the timed region)
# ----------------------------------------------------------------------------------------------

class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-lms", "100", "-i", str(self.index)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            time.sleep(0.3)
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.time(), line.strip()))

    def stop(self, t0, t1):
        if not self.proc:
            return None
        time.sleep(0.15)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], None, set()
        for ts, line in self.lines:
            if ts < t0 or ts > t1 + 0.1:
                continue
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for name, val in zip(("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"), f[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def jacobi_flops(m, n, info, rots, precond=False):
    """Algorithmic flops of one-sided Jacobi: every visited pair costs its 2x2 Gram (6 max(m,n)),
    every applied rotation 6(m + n) (A and V columns); sweeps = info (or info - NOT_CONVERGED).
    QR-preconditioned (square): plus the Householder factorisation 4n^3/3 and its application to
    the accumulated rotations 2n^3, per matrix."""
    info = np.asarray(info)
    sweeps = np.where(info >= (1 << 20), info - (1 << 20), info).astype(np.float64)
    k = min(m, n)
    mm = max(m, n)
    fl = float(np.sum(sweeps * (k * (k - 1) / 2) * 6 * mm + np.asarray(rots, np.float64) * 6 * (m + n)))
    if precond:
        fl += len(info) * (4.0 * n ** 3 / 3 + 2.0 * n ** 3)
    return fl


def block_jacobi_launches(n_cols, bw=32, sweeps=20):
    """Kernels one batched_svd_block_jacobi call launches (GRAM): setup, then for every sweep up to
    the cap -- launched whether or not matrices have converged, whose items the device lists then
    skip -- (blocks - 1) steps of Gram, inner SVD, polish and update plus the sweep-end kernel,
    then finalize."""
    nblk = max(2, -(-n_cols // bw))
    nblk += nblk & 1
    return 1 + sweeps * ((nblk - 1) * 4 + 1) + 1


def block_qr_launches(n_cols, bw=32, sweeps=20):
    """Kernels of a QR-preconditioned block-Jacobi call: setup, per 32-column panel the panel kernel
    and (but the last) the trailing update, R^T, the block Jacobi on R^T, the left vectors' zero
    fill and one block-reflector application per panel."""
    p = -(-n_cols // 32)
    return 1 + p + (p - 1) + 1 + block_jacobi_launches(n_cols, bw, sweeps) + 1 + p


def rsvd_launches(max_m, max_n, rounds):
    """Kernels one batched_rsvd call launches: plan and scan; per round the arrays kernel, the
    sampling GEMM, the QRs of the sample, the power step's two products and two QRs, the projection
    and its QR (each QR once per size bin the bounds can populate: rows in (0, 64], (64, 128],
    (128, ...), columns in (0, 32], (32, 64], (64, ...), no bin with more columns than rows), the
    small SVD per column bin (register tier; the shared tier for samples in (64, 128] and above), two
    GEMMs for U and V and the estimate; then the fallback and arrays kernels, the full-rank QR path
    (QR per row bin and column bin up to 128, the SVD of R^T per register-tier column bin and in the
    shared tier when min > 64, GEMM, copy), the block tier on R^T of a blocked QR (min > 128) and
    the finish kernel."""
    kx = min(max_m, max_n)
    lx = min(kx, 160)  # the FP32 sample cap

    def bins(rows_max, cols_max, col_bins):
        n = 0
        for rb in range(3):
            if rb > 0 and (64 << (rb - 1)) >= rows_max:
                break
            rbd = (64 << rb) if rb < 2 and (64 << rb) < rows_max else rows_max
            for cb in range(col_bins):
                if cb > 0 and (32 << (cb - 1)) >= cols_max:
                    break
                if cb > 0 and (32 << (cb - 1)) >= rbd:
                    continue  # no block has more samples than rows
                n += 1
        return n

    qy, qz = bins(max_m, lx, 3), bins(max_n, lx, 3)
    small = 1 + (1 if lx > 32 else 0)
    per_round = 1 + 1 + qy + (qz + 1 + qy + 1) + (1 + qz) + small + (1 if lx > 64 else 0) + (1 if lx > 128 else 0) + 2 + 1
    n = 2 + rounds * per_round + 2
    if kx > 0:
        kq = min(kx, 128)
        n += bins(max(max_m, max_n), kq, 3) + (1 + (1 if kq > 32 else 0)) + (1 if kq > 64 else 0) + 2
        n += block_qr_launches(kx) if kx > 128 else 0
    return n + 1


def tier_precond(bs, code, m, n, tier):
    """True when the encoded register tier is a QR-preconditioned variant."""
    if (tier & 0xff) != bs.TIER_REGISTER:
        return False
    k = tier >> 8 or 1
    return bool(bs.jacobi_variant_desc(code, m, n, k)["qr_precond"])


def max_over_ranks(x, world, dev):
    if world == 1:
        return x
    import torch
    t = torch.tensor([x], device=dev, dtype=torch.float64)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


# ----------------------------------------------------------------------------------------------
# workloads
# ----------------------------------------------------------------------------------------------

class SvdQr64:
    """20000 x (64 x 64) FP32 Jacobi SVD + 20000 x (128 x 32) FP32 QR per GPU per step."""
    name = "svd64_qr128"
    metric = "batched SVDs/s (64x64 FP32 Jacobi SVD + 128x32 FP32 QR per SVD)"
    unit = "SVDs/s"
    dtype = "f32"

    def __init__(self, args):
        self.args = args
        self.nb, self.nq = args.svd_batch, args.qr_batch

    def config(self, world):
        mb = (self.nb * 64 * 64 + self.nq * 128 * 32) * 4 / 1e6
        return {"workload": f"svd64_qr128: Jacobi SVD (U,S,V) of {self.nb} FP32 64x64 + Householder QR (Q,R) of "
                            f"{self.nq} FP32 128x32 per GPU per step; sigma_i = exp(-i/8), Haar U, V",
                "svd_batch_per_gpu": self.nb, "qr_batch_per_gpu": self.nq, "m": 64, "n": 64, "qr_m": 128,
                "qr_n": 32, "l2": f"inputs ({mb:.0f} MB per GPU) {'larger' if mb > 129 else 'smaller'} than L2; "
                                  "no flush",
                "parallelism": f"independent batches per GPU x{world}"}

    def setup(self, rank, dev):
        import torch
        import gen
        import paper_1707_05141_gb300 as bs
        from paper_1707_05141_gb300 import autotune
        self.bs = bs
        a_svd = gen.svd64_exp8(batch=self.nb, first=rank * self.nb)
        a_qr = gen.qr128x32_exp8(batch=self.nq, first=rank * self.nq)
        self.h_in = [torch.from_numpy(a_svd.a).pin_memory(), torch.from_numpy(a_qr.a).pin_memory()]
        self.d_svd, self.d_qr = (h.to(dev) for h in self.h_in)
        m = n = k = 64
        self.A = bs.Batch.uniform(self.d_svd, m, n)
        self.S = torch.empty((self.nb, 1, k), device=dev)
        self.U = torch.empty((self.nb, k, m), device=dev)
        self.V = torch.empty((self.nb, k, n), device=dev)
        self.Sb, self.Ub, self.Vb = bs.Batch.uniform(self.S, k, 1), bs.Batch.uniform(self.U, m, k), bs.Batch.uniform(self.V, n, k)
        self.info = torch.empty(self.nb, dtype=torch.int32, device=dev)
        self.rots = torch.empty(self.nb, dtype=torch.int64, device=dev)
        self.AQ = bs.Batch.uniform(self.d_qr, 128, 32)
        self.Q = torch.empty((self.nq, 32, 128), device=dev)
        self.R = torch.empty((self.nq, 32, 32), device=dev)
        self.Qb, self.Rb = bs.Batch.uniform(self.Q, 128, 32), bs.Batch.uniform(self.R, 32, 32)
        self.qinfo = torch.empty(self.nq, dtype=torch.int32, device=dev)
        if getattr(self.args, "jacobi_tier", None):
            # a given register variant instead of the autotuner's choice (profiling runs)
            t = int(self.args.jacobi_tier, 0)
            bs.set_jacobi_choice(bs.F32, m, n, t)
            self.tuned = {"tier": t, "ms": None, "sample": 0, "all_ms": {}, "forced": True}
        else:
            self.tuned = autotune.tune_jacobi(self.d_svd, m, n)
        self.outs = [self.S, self.U, self.V, self.Q, self.R]
        self.d_in = [self.d_svd, self.d_qr]
        self.qr_ev = []  # (before, after) the QR launch of every timed step

    def step(self, stream, kev=None):
        if kev is not None:
            import torch
            e = torch.cuda.Event(enable_timing=True)
            e.record(stream)
            self.qr_ev.append((e, kev[0]))
        self.bs.batched_qr(self.AQ, self.Qb, self.Rb, self.qinfo, stream)
        if kev is not None:
            kev[0].record(stream)
        self.bs.batched_svd_jacobi(self.A, self.Sb, self.Ub, self.Vb, self.info, self.rots, stream=stream)
        if kev is not None:
            kev[1].record(stream)

    launches_per_step = 2
    units = property(lambda self: self.nb)

    def host_step(self, houts, chunks):
        """One end-to-end step through the host entries: QR then SVD of the host batches, outputs to
        the pinned host buffers (S, U, V, Q, R)."""
        import torch
        bs = self.bs
        dev = self.d_svd.device
        h_svd, h_qr = self.h_in
        hs, hu, hv, hq, hr = houts
        ws_q = torch.empty(bs.host_qr_workspace(bs.F32, self.nq, 128, 32), dtype=torch.uint8, device=dev)
        ws_s = torch.empty(bs.host_svd_workspace(bs.F32, self.nb, 64, 64), dtype=torch.uint8, device=dev)

        side = torch.cuda.Stream(device=dev)

        def step(stream):
            # the two independent calls on two streams: the QR's copies and kernels overlap the
            # SVD's (the library's copy streams keep each direction's transfers in issue order)
            side.wait_stream(stream)
            bs.host_qr(h_qr, hq, hr, chunks=chunks, workspace=ws_q, stream=side)
            bs.host_svd(h_svd, hs, hu, hv, chunks=chunks, workspace=ws_s, stream=stream)
            stream.wait_stream(side)
        return step

    def roofline(self, kernel_ms):
        bs = self.bs
        info_h, rots_h = self.info.cpu().numpy(), self.rots.cpu().numpy()
        assert np.all(info_h > 0), "Jacobi reported a bad shape"
        pre = tier_precond(bs, bs.F32, 64, 64, int(self.tuned["tier"]))
        fl = jacobi_flops(64, 64, info_h, rots_h, pre)
        achieved = fl / (kernel_ms * 1e-3) / 1e12
        tier = int(self.tuned["tier"])
        reg = (tier & 0xff) == bs.TIER_REGISTER
        kname = ("jacobi_reg_kernel" if reg else "jacobi_smem_kernel") + f" (tier {tier:#x})"
        traffic = TRAFFIC.get("jacobi_reg:" + kernel_digest("jacobi_reg.cu")) if reg else None
        if traffic is not None:
            traffic *= self.nb / 20000  # per launch: scales with the matrix count
        roof = {"kernel": kname, "bound": "alu", "achieved": achieved, "peak": PEAKS["fp32"]["tflops"], "unit": "TFLOP/s",
                "frac": achieved / PEAKS["fp32"]["tflops"], "traffic": traffic, "ms_per_launch": kernel_ms,
                "peak_note": PEAKS["fp32"]["note"]}
        detail = {"svd_sweeps_mean": float(np.mean(info_h)), "rotations_mean": float(np.mean(rots_h)),
                  "jacobi_gflop_per_launch": fl / 1e9, "autotune": self.tuned}
        if self.qr_ev:
            # the QR launch: HBM-bound, one read of A and the Q, R writes per matrix
            qr_ms = statistics.mean(a.elapsed_time(b) for a, b in self.qr_ev)
            qbytes = self.nq * (128 * 32 * 2 + 32 * 32) * 4
            gbs = qbytes / (qr_ms * 1e-3) / 1e9
            peak = measured_hbm_gbs()
            qtraffic = TRAFFIC.get("qr:" + kernel_digest("qr.cu"))
            detail["qr"] = {"kernel": "qr_warp_kernel<float, 128, 1>", "ms_per_launch": qr_ms,
                            "bytes_per_launch": qbytes, "achieved_gbs": gbs, "peak_gbs": peak,
                            "frac": gbs / peak, "bound": "hbm", "peak_note": "measured copy bandwidth",
                            "traffic": qtraffic * self.nq / 20000 if qtraffic is not None else None}
            self.qr_ev = []
        return roof, detail

    def extra_arms(self, stream, steps, warmup, time_fn):
        """The register variant of the tuned one's shape (carried norms off) with its rotation
        parameters (zeta, t, c, s) and rotation test in FP32, and the same with them in FP64 from the
        FP32 Gram sums: the cost of the FP64 parameters, measured side by side."""
        import torch
        bs = self.bs
        tier = int(self.tuned["tier"])
        if (tier & 0xff) != bs.TIER_REGISTER:
            return {}
        base = dict(bs.jacobi_variant_desc(bs.F32, 64, 64, tier >> 8 or 1), carried_norms=0)
        nv = bs.jacobi_variants(bs.F32, 64, 64, bs.TIER_REGISTER)
        descs = {k: bs.jacobi_variant_desc(bs.F32, 64, 64, k) for k in range(1, nv + 1)}
        k32 = next((k for k, d in descs.items() if d == dict(base, fp64_params=0)), None)
        k64 = next((k for k, d in descs.items() if d == dict(base, fp64_params=1)), None)
        if k32 is None or k64 is None:
            return {}
        out = {}
        for name, k in (("fp32", k32), ("fp64", k64)):
            t_k = bs.TIER_REGISTER | (k << 8)

            def step(st, kev=None, t_k=t_k):
                if kev is not None:
                    kev[0].record(st)
                bs.batched_svd_jacobi(self.A, self.Sb, self.Ub, self.Vb, self.info, self.rots, tier=t_k, stream=st)
                if kev is not None:
                    kev[1].record(st)
            for _ in range(warmup):
                step(stream)
            torch.cuda.synchronize()
            t = time_fn(step)
            info_h, rots_h = self.info.cpu().numpy(), self.rots.cpu().numpy()
            fl = jacobi_flops(64, 64, info_h, rots_h, bool(base["qr_precond"]))
            achieved = fl / (t["kernel_ms"] * 1e-3) / 1e12
            out[name] = {"tier": hex(t_k), "ms_per_launch": t["kernel_ms"], "clocks": t["clocks"],
                         "achieved_tflops": achieved, "frac": achieved / PEAKS["fp32"]["tflops"],
                         "svd_sweeps_mean": float(np.mean(info_h))}
        out["slowdown"] = out["fp64"]["ms_per_launch"] / out["fp32"]["ms_per_launch"]
        return {"rotation_parameter_precision": out}

    def cpu_sample(self, n):
        import gen
        import oracle
        a_svd = gen.svd64_exp8(batch=n)
        a_qr = gen.qr128x32_exp8(batch=n)
        cores = oracle.default_threads()
        mats, qmats = [a_svd.a64(i) for i in range(n)], [a_qr.a64(i) for i in range(n)]
        t0 = time.time()
        oracle.svd_batch(mats, nthreads=cores)
        oracle.qr_batch(qmats, nthreads=cores)
        dt = time.time() - t0
        return {"value": n / dt, "count": n, "seconds": dt, "unit": self.unit, "cores": cores, "kind": "oracle",
                "sample": f"{n} SVDs of 64x64 + {n} QRs of 128x32 (same generator), FP64, {dt:.2f} s wall"}


class Fp64_32:
    """1000 x (32 x 32) FP64 Jacobi SVD + QR of the same matrices."""
    name = "fp64_32"
    metric = "batched SVDs/s (32x32 FP64 Jacobi SVD + 32x32 FP64 QR per SVD)"
    unit = "SVDs/s"
    dtype = "f64"
    launches_per_step = 2
    flush_l2 = True  # the 8 MB batch fits in L2

    def __init__(self, args):
        self.args = args
        self.nb = 1000

    def config(self, world):
        return {"workload": "fp64_32: Jacobi SVD (U,S,V) and Householder QR of 1000 FP64 32x32 per GPU per step; "
                            "sigma_i = 10^(-8 i/31)", "batch_per_gpu": self.nb,
                "l2": "8 MB inputs fit in L2: a 256 MB write flushes L2 before every timed step, outside that "
                      "step's events (ms_per_step sums the steps' own events)",
                "parallelism": f"independent batches per GPU x{world}"}

    def setup(self, rank, dev):
        import torch
        import gen
        import paper_1707_05141_gb300 as bs
        from paper_1707_05141_gb300 import autotune
        self.bs = bs
        b = gen.fp64_32_graded(batch=self.nb, first=rank * self.nb)
        self.h_in = [torch.from_numpy(b.a).pin_memory()]
        self.d = self.h_in[0].to(dev)
        self.d_in = [self.d]
        k = 32
        self.A = bs.Batch.uniform(self.d, 32, 32)
        self.S = torch.empty((self.nb, 1, k), device=dev, dtype=torch.float64)
        self.U = torch.empty((self.nb, k, 32), device=dev, dtype=torch.float64)
        self.V = torch.empty((self.nb, k, 32), device=dev, dtype=torch.float64)
        self.Q = torch.empty((self.nb, 32, 32), device=dev, dtype=torch.float64)
        self.R = torch.empty((self.nb, 32, 32), device=dev, dtype=torch.float64)
        self.Sb, self.Ub, self.Vb = (bs.Batch.uniform(self.S, k, 1), bs.Batch.uniform(self.U, 32, k),
                                     bs.Batch.uniform(self.V, 32, k))
        self.Qb, self.Rb = bs.Batch.uniform(self.Q, 32, 32), bs.Batch.uniform(self.R, 32, 32)
        self.info = torch.empty(self.nb, dtype=torch.int32, device=dev)
        self.qinfo = torch.empty(self.nb, dtype=torch.int32, device=dev)
        self.rots = torch.empty(self.nb, dtype=torch.int64, device=dev)
        self.tuned = autotune.tune_jacobi(self.d, 32, 32, sample=self.nb)
        self.outs = [self.S, self.U, self.V, self.Q, self.R]

    def step(self, stream, kev=None):
        self.bs.batched_qr(self.A, self.Qb, self.Rb, self.qinfo, stream)
        if kev is not None:
            kev[0].record(stream)
        self.bs.batched_svd_jacobi(self.A, self.Sb, self.Ub, self.Vb, self.info, self.rots, stream=stream)
        if kev is not None:
            kev[1].record(stream)

    units = property(lambda self: self.nb)

    def host_step(self, houts, chunks):
        """One end-to-end step through the host entries: QR and SVD of the host batch (one chunk:
        a quarter of this 1000-matrix batch no longer fills the GPU)."""
        import torch
        bs = self.bs
        dev = self.d.device
        h_a = self.h_in[0]
        hs, hu, hv, hq, hr = houts
        ws_q = torch.empty(bs.host_qr_workspace(bs.F64, self.nb, 32, 32), dtype=torch.uint8, device=dev)
        ws_s = torch.empty(bs.host_svd_workspace(bs.F64, self.nb, 32, 32), dtype=torch.uint8, device=dev)

        def step(stream):
            bs.host_qr(h_a, hq, hr, chunks=1, workspace=ws_q, stream=stream)
            bs.host_svd(h_a, hs, hu, hv, chunks=1, workspace=ws_s, stream=stream)
        return step

    def roofline(self, kernel_ms):
        info_h, rots_h = self.info.cpu().numpy(), self.rots.cpu().numpy()
        pre = tier_precond(self.bs, self.bs.F64, 32, 32, int(self.tuned["tier"]))
        fl = jacobi_flops(32, 32, info_h, rots_h, pre)
        achieved = fl / (kernel_ms * 1e-3) / 1e12
        return ({"kernel": f"jacobi_reg_kernel<double> (tier {int(self.tuned['tier']):#x})", "bound": "alu",
                 "achieved": achieved, "peak": PEAKS["fp64"]["tflops"], "unit": "TFLOP/s",
                 "frac": achieved / PEAKS["fp64"]["tflops"], "traffic": None, "ms_per_launch": kernel_ms,
                 "peak_note": PEAKS["fp64"]["note"]},
                {"svd_sweeps_mean": float(np.mean(info_h)), "rotations_mean": float(np.mean(rots_h)),
                 "autotune": self.tuned})

    def cpu_sample(self, n):
        import gen
        import oracle
        b = gen.fp64_32_graded(batch=n)
        mats = [b.a64(i) for i in range(n)]
        cores = oracle.default_threads()
        t0 = time.time()
        oracle.svd_batch(mats, nthreads=cores)
        oracle.qr_batch(mats, nthreads=cores)
        dt = time.time() - t0
        return {"value": n / dt, "count": n, "seconds": dt, "unit": self.unit, "cores": cores, "kind": "oracle",
                "sample": f"{n} SVDs + QRs of 32x32 FP64 (same generator), {dt:.2f} s wall"}


class Block512:
    """500 x (512 x 512) FP32 block-Jacobi SVD (GRAM, block width 32)."""
    name = "block512"
    metric = "batched SVDs/s (512x512 FP32 block-Jacobi SVD)"
    unit = "SVDs/s"
    dtype = "f32"
    launches_per_step = block_qr_launches(512, 32, 20)   # every sweep up to the cap of 20 is launched

    def __init__(self, args):
        self.args = args
        self.nb = args.block_batch

    def config(self, world):
        return {"workload": f"block512: block-Jacobi SVD (U,S,V) of {self.nb} FP32 512x512 per GPU per step, blocked "
                            "Householder QR then GRAM block Jacobi on R^T (block width and inner pair SVD by the autotuner, pair "
                            "Gram products on the tensor cores for width 32: TF32 hi/lo split, FP32 accumulation; updates on "
                            "FP32 SIMT), U = Q V~; "
                            "sigma log-uniform on [1e-6, 1]", "batch_per_gpu": self.nb,
                "l2": f"inputs ({self.nb * 512 * 512 * 4 / 1e6:.0f} MB per GPU) "
                      f"{'larger' if self.nb * 512 * 512 * 4 > 129e6 else 'smaller'} than L2",
                "parallelism": f"independent batches per GPU x{world}"}

    def setup(self, rank, dev):
        import torch
        import gen
        import paper_1707_05141_gb300 as bs
        self.bs = bs
        if self.args.host_inputs:
            b = gen.block512_loguniform(batch=self.nb, first=rank * self.nb)
            self.h_in = [torch.from_numpy(b.a).pin_memory()]
            self.d = self.h_in[0].to(dev)
            self.sigma = b.sigma
        else:  # the same recipe generated on the device (minutes of host LAPACK time otherwise)
            from gen import device as gdev
            self.d, self.sigma = gdev.block512_loguniform(batch=self.nb, first=rank * self.nb, dev=dev)
            self.h_in = None
        self.d_in = [self.d]
        k = 512
        self.A = bs.Batch.uniform(self.d, 512, 512)
        self.S = torch.empty((self.nb, 1, k), device=dev)
        self.U = torch.empty((self.nb, k, 512), device=dev)
        self.V = torch.empty((self.nb, k, 512), device=dev)
        self.Sb, self.Ub, self.Vb = (bs.Batch.uniform(self.S, k, 1), bs.Batch.uniform(self.U, 512, k),
                                     bs.Batch.uniform(self.V, 512, k))
        self.info = torch.empty(self.nb, dtype=torch.int32, device=dev)
        self.rots = torch.empty(self.nb, dtype=torch.int64, device=dev)
        # block width and inner pair-SVD variant by the autotuner (block_width = 0 uses its choice)
        from paper_1707_05141_gb300 import autotune
        self.tuned = autotune.tune_block(self.d, method=bs.BLOCK_QR_PRECONDITION, sample=min(64, self.nb))
        self.bw = int(self.tuned["block_width"])
        self.ws = torch.empty(max(bs.batched_svd_block_jacobi_workspace(self.A, 0, m)
                                  for m in (0, bs.BLOCK_QR_PRECONDITION, bs.BLOCK_SIMT_PRODUCTS)),
                              dtype=torch.uint8, device=dev)
        self.outs = [self.S, self.U, self.V]

    def step(self, stream, kev=None):
        if kev is not None:
            kev[0].record(stream)
        self.bs.batched_svd_block_jacobi(self.A, self.Sb, self.Ub, self.Vb, self.info, self.ws, self.rots,
                                         max_sweeps=20, block_width=0, method=self.bs.BLOCK_QR_PRECONDITION,
                                         stream=stream)
        if kev is not None:
            kev[1].record(stream)

    mixed_form = ("blocked Householder QR, GRAM block Jacobi on R^T with the pair Gram products on the tensor cores "
                  "(tcgen05 TF32 hi/lo split, FP32 accumulation), U = Q V~")
    plain_form = "pair Gram products on the FP32 SIMT pipes (BSVD_BLOCK_SIMT_PRODUCTS)"

    def quality(self):
        info_h = self.info.cpu().numpy()
        sweeps = np.where(info_h >= (1 << 20), info_h - (1 << 20), info_h)
        s = self.S.cpu().numpy()[:, 0, :].astype(np.float64)
        err = float(np.max(np.abs(s - self.sigma).max(axis=1) / self.sigma[:, 0]))
        return {"sweeps_mean": float(np.mean(sweeps)), "max_sigma_err_vs_generator_normwise": err,
                "within_1e-5": bool(err <= 1e-5)}

    def _step_fn(self, method):
        def step(st, kev=None):
            if kev is not None:
                kev[0].record(st)
            self.bs.batched_svd_block_jacobi(self.A, self.Sb, self.Ub, self.Vb, self.info, self.ws, self.rots,
                                             max_sweeps=20, block_width=0, method=method, stream=st)
            if kev is not None:
                kev[1].record(st)
        return step

    def plain_arm(self, stream):
        return self._step_fn(self.bs.BLOCK_SIMT_PRODUCTS), self.quality

    def extra_arms(self, stream, steps, warmup, time_fn):
        """GRAM on A itself (no QR preconditioning), tensor-core Gram; and the default form with every
        block pair re-tested every sweep (no pair selection by the recorded tests)."""
        import torch
        out = {}
        for name, method, form in (
                ("no_qr_preconditioning", 0, "GRAM block Jacobi on A (tensor-core Gram), no QR preconditioning"),
                ("retest_every_pair", self.bs.BLOCK_QR_PRECONDITION | self.bs.BLOCK_RETEST_ALL,
                 "the default form re-testing every block pair every sweep (BSVD_BLOCK_RETEST_ALL): the "
                 "recorded pair tests skip pairs found orthogonal whose blocks did not change since")):
            step = self._step_fn(method)
            for _ in range(warmup):
                step(stream)
            torch.cuda.synchronize()
            t = time_fn(step)
            out[name] = {"form": form, "ms_per_step": t["ms_step"], "clocks": t["clocks"],
                         "value": self.units / (t["ms_step"] * 1e-3), **self.quality()}
        return out

    units = property(lambda self: self.nb)

    def roofline(self, kernel_ms):
        info_h = self.info.cpu().numpy()
        sweeps = np.where(info_h >= (1 << 20), info_h - (1 << 20), info_h)
        # per pair: Gram 2 m (2bw)^2, update 2 (m + n) (2bw)^2 flops; nb (nb - 1) / 2 pairs per sweep
        # (nb = 512 / bw blocks); per matrix the blocked QR (4 n^3 / 3) and U = Q V~ (2 n^3)
        k2 = 2 * self.bw
        nblk = 512 // self.bw
        pair_fl = 2 * 512 * k2 * k2 + 2 * 1024 * k2 * k2
        fl = float(np.sum(sweeps) * (nblk * (nblk - 1) // 2) * pair_fl) + self.nb * (4.0 / 3.0 + 2.0) * 512 ** 3
        achieved = fl / (kernel_ms * 1e-3) / 1e12
        return ({"kernel": "batched_svd_block_jacobi (all stages of one call)", "bound": "alu",
                 "achieved": achieved, "peak": PEAKS["fp32"]["tflops"], "unit": "TFLOP/s",
                 "frac": achieved / PEAKS["fp32"]["tflops"], "traffic": None, "ms_per_launch": kernel_ms,
                 "peak_note": PEAKS["fp32"]["note"] + "; achieved counts Gram + update flops of the pairs of "
                              "every sweep run, the blocked QR and U = Q V~"},
                {"sweeps_max": int(np.max(sweeps)), "autotune": self.tuned, **self.quality()})

    def cpu_sample(self, n):
        import oracle
        n = max(1, min(n, 16, self.nb))
        a = self.d[:n].cpu().numpy()
        mats = [a[i].T.astype(np.float64) for i in range(n)]
        cores = oracle.default_threads()
        t0 = time.time()
        oracle.svd_batch(mats, nthreads=cores)
        dt = time.time() - t0
        return {"value": n / dt, "count": n, "seconds": dt, "unit": self.unit, "cores": cores, "kind": "oracle",
                "sample": f"{n} SVDs of 512x512 FP64 (the first matrices of the timed batch), {dt:.2f} s wall"}


class DeviceBlocks:
    """Uneven blocks generated on the device, with a pinned host copy for the end-to-end run, the
    error checks and the oracle's sample."""

    def __init__(self, flat_d, offset, m, n, extra):
        self.flat_d = flat_d
        self.h = flat_d.cpu().pin_memory()
        self.flat = self.h.numpy()
        self.offset, self.m, self.n, self.extra = offset, m, n, extra

    @property
    def batch(self):
        return len(self.m)

    def a64(self, b):
        mb, nb, o = int(self.m[b]), int(self.n[b]), int(self.offset[b])
        return self.flat[o:o + mb * nb].reshape(nb, mb).T.astype(np.float64)


class RsvdBase:
    unit = "SVDs/s"
    dtype = "f32"
    flags = 0   # the timed form samples in FP32 (the tensor-core sample is an arm: measured slower)

    def _alloc(self, rb, dev, hint_host):
        import torch
        bs = self.bs
        self.rb = rb
        m, n = rb.m, rb.n
        k = np.minimum(m, n)
        if getattr(rb, "flat_d", None) is not None:   # generated on the device
            self.h_in = [rb.h]
            self.flat = rb.flat_d
        else:
            self.h_in = [torch.from_numpy(rb.flat).pin_memory()]
            self.flat = self.h_in[0].to(dev)
        self.d_in = [self.flat]
        su, sv, ss = (m.astype(np.int64) * k + 3) // 4 * 4, (n.astype(np.int64) * k + 3) // 4 * 4, (k + 3) // 4 * 4
        off = lambda x: np.concatenate([[0], np.cumsum(x)[:-1]])
        self.fu = torch.zeros(int(su.sum()), device=dev)
        self.fv = torch.zeros(int(sv.sum()), device=dev)
        self.fs = torch.zeros(int(ss.sum()), device=dev)
        self.A = bs.Batch.packed(self.flat, rb.offset, m, n)
        self.U = bs.Batch.packed(self.fu, off(su), m, k)
        self.V = bs.Batch.packed(self.fv, off(sv), n, k)
        self.S = bs.Batch.packed(self.fs, off(ss), k, np.ones_like(k))
        self.kmax = torch.as_tensor(k.astype(np.int32)).to(dev)
        self.rank = torch.zeros(rb.batch, dtype=torch.int32, device=dev)
        self.info = torch.zeros(rb.batch, dtype=torch.int32, device=dev)
        self.err = torch.zeros(rb.batch, dtype=torch.float32, device=dev)
        self.samples = torch.zeros(rb.batch, dtype=torch.int32, device=dev)
        self.ws = torch.empty(bs.batched_rsvd_workspace(self.A, m, n), dtype=torch.uint8, device=dev)
        self.hint = None if hint_host is None else torch.as_tensor(np.asarray(hint_host, np.int32)).to(dev)
        self.outs = [self.fu, self.fv, self.fs]
        self.graph = None

    def _rsvd(self, stream, hint, rounds, fixed=None, flags=0):
        self.bs.batched_rsvd(self.A, self.U, self.S, self.V, self.kmax, self.rank, self.info, self.ws, hint,
                             tol=1e-5, oversample=8, max_rounds=rounds, seed=1707, err_est=self.err,
                             samples=self.samples, stream=stream, fixed_rank=fixed, flags=flags)

    def _timed_arm(self, fn, stream, warmup, time_fn, form):
        import torch
        step = self._graph_arm(fn)
        for _ in range(warmup):
            step(stream)
        torch.cuda.synchronize()
        t = time_fn(step)
        return {"form": form, "ms_per_step": t["ms_step"], "clocks": t["clocks"],
                "value": self.units / (t["ms_step"] * 1e-3), **self.quality()}

    def extra_arms(self, stream, steps, warmup, time_fn):
        """The timed form with the small SVDs in FP64 as well (BSVD_RSVD_SMALL_FP64: the precision
        split of the method -- low-precision sample, FP64 small SVD), and with FP32 sampling."""
        bs = self.bs
        return {"small_svd_fp64": self._timed_arm(
                    lambda st: self.inner(st, self.flags | bs.RSVD_SMALL_FP64), stream, warmup, time_fn,
                    self.mixed_form + "; small SVDs in FP64"),
                "tc_sampling": self._timed_arm(
                    lambda st: self.inner(st, self.flags | bs.RSVD_TC_SAMPLING), stream, warmup, time_fn,
                    self.mixed_form + "; sample A Omega on the tensor cores (tcgen05 kind::tf32, FP32 "
                                      "accumulation; probes in FP32)")}

    def _graph_arm(self, fn):
        """A step function replaying a CUDA graph of fn(stream) (captured now)."""
        import torch
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            fn(torch.cuda.current_stream())

        def step(stream, kev=None):
            if kev is not None:
                kev[0].record(stream)
            g.replay()
            if kev is not None:
                kev[1].record(stream)
        step.graph = g
        return step

    plain_form = "FP32 SIMT sampling and projection, adaptive range finder from 8 samples (no rank hints)"

    def plain_arm(self, stream):
        return self._graph_arm(lambda st: self._rsvd(st, None, 16)), self.quality

    def quality(self):
        info = self.info.cpu().numpy()
        samp = self.samples.cpu().numpy()
        err = self.error_sample()
        return {"rounds_mean": float((info & 0xff).mean()), "samples_mean": float(samp.mean()),
                "fallback_frac": float(np.mean((info >> 22) & 1)), "rank_mean": float(self.rank.float().mean()),
                "max_rel_error_sampled": err, "within_1e-5": bool(err <= 1e-5)}

    def capture(self, stream):
        import torch
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):          # captured on torch's side stream
            self.inner(torch.cuda.current_stream())

    def step(self, stream, kev=None):
        if kev is not None:
            kev[0].record(stream)
        if self.graph is not None:
            self.graph.replay()
        else:
            self.inner(stream)
        if kev is not None:
            kev[1].record(stream)

    units = property(lambda self: self.rb.batch)

    def error_sample(self, nsamp=64):
        """Relative truncation error ||A - U_k S_k V_k^T||_F / ||A||_F on sampled blocks (FP64, host)."""
        rb = self.rb
        U, V, S = (t.cpu().numpy().astype(np.float64) for t in (self.fu, self.fv, self.fs))
        rk = self.rank.cpu().numpy()
        ou, ov, os_ = (np.asarray(x.ptrs.cpu().numpy() - x.ptrs[0].item(), np.int64) // 4 for x in (self.U, self.V, self.S))
        worst = 0.0
        for b in range(0, rb.batch, max(1, rb.batch // nsamp)):
            a = rb.a64(b)
            m, n, k = a.shape[0], a.shape[1], int(rk[b])
            u = U[ou[b]:ou[b] + m * k].reshape(k, m).T
            v = V[ov[b]:ov[b] + n * k].reshape(k, n).T
            s = S[os_[b]:os_[b] + k]
            worst = max(worst, float(np.linalg.norm(a - (u * s) @ v.T) / np.linalg.norm(a)))
        return worst

    def roofline(self, kernel_ms):
        info = self.info.cpu().numpy()
        rounds = info & 0xff
        samp = self.samples.cpu().numpy()
        rb = self.rb
        # algorithmic bytes: one read of A plus the writes of U, S, V of rank k (the method's
        # minimum when a block is factored on chip); the secondary count takes every pass over A
        # the method makes (sample, two power-step products, projection per round; one per full SVD)
        rk = self.rank.cpu().numpy().astype(np.float64)
        outb = float(np.sum((rb.m + rb.n + 1) * rk * 4))
        abytes = float(np.sum(rb.m.astype(np.float64) * rb.n * 4)) + outb
        pbytes = float(np.sum((rb.m.astype(np.float64) * rb.n) * 4 * (4 * rounds + (samp == np.minimum(rb.m, rb.n))))) + outb
        achieved = abytes / (kernel_ms * 1e-3) / 1e9
        passes_gbs = pbytes / (kernel_ms * 1e-3) / 1e9
        peak = measured_hbm_gbs()
        k = np.minimum(rb.m, rb.n)
        return ({"kernel": self.kernel_name, "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                 "frac": achieved / peak, "traffic": None, "ms_per_launch": kernel_ms,
                 "peak_note": "measured copy bandwidth (MEASURED_PEAKS.json); achieved = algorithmic bytes "
                              "(one read of A + the writes of U, S, V of rank k) of the whole call / its time",
                 "achieved_passes": passes_gbs, "passes_note": "the same time against the bytes of every pass "
                 "the method makes over A (four per sampling round, one per full SVD) plus the outputs"},
                {"full_rank_frac": float(np.mean(samp == k)), **self.quality()})

    def cpu_sample_blocks(self, rb, n, hint):
        import oracle
        cores = oracle.default_threads()
        idx = list(range(0, rb.batch, max(1, rb.batch // n)))[:n]
        from concurrent.futures import ThreadPoolExecutor

        def one(b):
            oracle.rsvd_adaptive(rb.a64(b), 1707, b, int(hint[b]) if hint is not None else 0, 1e-5, 8, 1, 16, 160)

        t0 = time.time()
        with ThreadPoolExecutor(max_workers=cores) as ex:
            list(ex.map(one, idx))
        dt = time.time() - t0
        return len(idx), dt, cores


class RsvdUneven(RsvdBase):
    name = "rsvd_uneven"
    metric = "batched randomized SVDs/s at 1e-5 relative Frobenius error (uneven 64..256 blocks)"
    kernel_name = "batched_rsvd (whole call, CUDA graph)"

    def __init__(self, args):
        self.args = args
        self.nb = args.rsvd_batch

    def config(self, world):
        return {"workload": f"rsvd_uneven: randomized SVD to 1e-5 of {self.nb} FP32 blocks per GPU, m, n uniform on "
                            "{64, 128, 256}, sigma_i = exp(-i/r0), r0 ~ U[2, 12]; p = 8, one power step, rank hint "
                            "= the rank where sigma falls to 1e-5; one CUDA graph per step",
                "batch_per_gpu": self.nb, "l2": f"inputs ({self.nb * 89335 / 1e9:.2f} GB per GPU on average) "
                f"{'larger' if self.nb * 89335 > 129e6 else 'smaller'} than L2",
                "parallelism": f"independent batches per GPU x{world}"}

    def setup(self, rank, dev):
        import gen
        import paper_1707_05141_gb300 as bs
        self.bs = bs
        if self.args.host_inputs:
            rb = gen.rsvd_uneven_blocks(batch=self.nb, first=rank * self.nb)
        else:  # the same recipe generated on the device (minutes of host LAPACK time otherwise)
            from gen import device as gdev
            flat, off, m, n, r0, hint = gdev.rsvd_uneven_blocks(batch=self.nb, first=rank * self.nb, dev=dev)
            rb = DeviceBlocks(flat, off, m, n, {"r0": r0, "rank_hint": hint})
        self._alloc(rb, dev, rb.extra["rank_hint"])
        self.kstar = self.hint

    def inner(self, stream, flags=None):
        self._rsvd(stream, self.hint, 4, flags=self.flags if flags is None else flags)

    mixed_form = ("tolerance mode with the rank where sigma falls to 1e-5 as the first guess, FP32 sampling, "
                  "one CUDA graph per step")

    def extra_arms(self, stream, steps, warmup, time_fn):
        """Plus fixed-rank mode (Algorithm 4 as stated) at k* = the rank where sigma falls to 1e-5."""
        out = super().extra_arms(stream, steps, warmup, time_fn)
        out["fixed_rank_kstar"] = self._timed_arm(lambda st: self._rsvd(st, None, 1, fixed=self.kstar), stream,
                                                  warmup, time_fn,
                                                  "fixed rank k* + 8 samples, one power step (Algorithm 4)")
        return out

    launches_per_step = rsvd_launches(256, 256, 4)

    def cpu_sample(self, n):
        rb = getattr(self, "rb", None)
        if rb is None:   # the reference arm: no device, the host generator
            import gen
            rb = gen.rsvd_uneven_blocks(batch=max(n, 1))
        cnt, dt, cores = self.cpu_sample_blocks(rb, n, rb.extra["rank_hint"])
        return {"value": cnt / dt, "count": cnt, "seconds": dt, "unit": self.unit, "cores": cores, "kind": "oracle",
                "sample": f"{cnt} blocks spread over the batch, FP64 adaptive RSVD (the oracle's range finder "
                          f"from hint + 8 columns, one power step, full Jacobi SVD fallback), {dt:.2f} s wall"}


class HmatrixMlp(RsvdBase):
    name = "hmatrix_mlp"
    metric = "batched randomized SVDs/s at 1e-5 with learned rank hints (kernel blocks)"
    kernel_name = "sketch features + MLP + batched_rsvd (whole step, CUDA graph)"

    def __init__(self, args):
        self.args = args

    def config(self, world):
        return {"workload": "hmatrix_mlp: admissible blocks (64..256) of exp(-|x-y|/0.1) over 32768 uniform 3D points "
                            "(k-d tree, median split, leaf 64, eta 1.1); randomized SVD to 1e-5 with ranks from the "
                            "rank predictor (trained on another point set's plain-adaptive ranks); plain adaptive "
                            "timed alongside", "blocks_per_gpu": getattr(self, "nblocks", None),
                "l2": "inputs (2.25 GB per GPU) larger than L2", "parallelism": f"independent point sets x{world}"}

    def setup(self, rank, dev):
        import torch
        import gen
        import paper_1707_05141_gb300 as bs
        from paper_1707_05141_gb300 import rank_mlp
        self.bs = bs
        self.rank_mlp = rank_mlp
        tr = gen.kernel_blocks_3d(n_points=16384, seed_index=100 + rank)
        ft = torch.from_numpy(tr.flat).to(dev)
        ranks, _ = rank_mlp.plain_adaptive_ranks(ft, tr.offset, tr.m, tr.n, seed=5)
        feats = rank_mlp.features(ft, tr.offset, tr.m, tr.n, seed=6)
        t0 = time.time()
        self.params, hist = rank_mlp.train(feats, ranks, steps=2000, log_every=500)
        self.train_info = {"train_blocks": tr.batch, "final_loss": hist[-1][1], "train_s": time.time() - t0}
        del ft, feats
        rb = gen.kernel_blocks_3d(n_points=32768, seed_index=rank)
        self.nblocks = rb.batch
        self._alloc(rb, dev, None)
        self.feats = torch.empty((rb.batch, 16), device=dev)
        self.pred = torch.empty(rb.batch, device=dev)
        self.hint_d = torch.empty(rb.batch, dtype=torch.int32, device=dev)
        self.md = torch.as_tensor(rb.m).to(dev)
        self.nd = torch.as_tensor(rb.n).to(dev)

    def inner(self, stream, flags=None):
        bs = self.bs
        bs.bsvd_sketch_features(self.A, self.feats, 6, stream)
        bs.bsvd_mlp_forward(self.feats, self.params, self.pred, self.hint_d, 2.0, self.md, self.nd, stream)
        self._rsvd(stream, self.hint_d, 16, flags=self.flags if flags is None else flags)

    launches_per_step = 2 + rsvd_launches(256, 256, 16)   # features, forward, then the randomized SVD

    mixed_form = "ranks predicted by the learned network (sketch features + MLP on the GPU) as first guesses"

    def cpu_sample(self, n):
        import gen
        rb = getattr(self, "_cpu_rb", None)
        if rb is None:  # generated once: every sample times the first n blocks of the same set
            rb = self._cpu_rb = gen.kernel_blocks_3d(n_points=8192, seed_index=0)
        cnt, dt, cores = self.cpu_sample_blocks(rb, n, None)
        return {"value": cnt / dt, "count": cnt, "seconds": dt, "unit": self.unit, "cores": cores, "kind": "oracle",
                "sample": f"{cnt} kernel blocks (8192-point set), FP64 adaptive RSVD from 8 columns (one power "
                          f"step, rounds of 8), {dt:.2f} s wall"}


class H2Truncation:
    """Truncation of an H^2 nested row basis (Section 8.2): Chebyshev-interpolation basis (q = 8,
    rank 64) over a k-d tree of depth 14 (mean split) on 2^20 points of a perturbed grid."""
    name = "h2_truncation"
    metric = "H2 basis-tree truncations/s (depth-14 Chebyshev basis, 16384 leaves, eps 1e-5)"
    unit = "trees/s"
    dtype = "f32"
    units = 1

    def __init__(self, args):
        self.args = args
        self.depth = getattr(args, "h2_depth", 14)

    def config(self, world):
        return {"workload": f"h2_truncation: truncation to eps 1e-5 of the Chebyshev-interpolation row basis (q = 8, "
                            f"rank 64) of a k-d tree of depth {self.depth} (mean split, {2 ** self.depth} leaves of "
                            "~64 points) over a perturbed grid of the unit square; FP32; leaf SVDs and one batched "
                            "SVD per level", "leaves": 2 ** self.depth,
                "l2": f"basis ({2 ** self.depth * 64 * 64 * 4 * 2 / 1e6:.0f} MB of leaves and transfers) "
                      f"{'larger' if 2 ** self.depth * 64 * 64 * 8 > 129e6 else 'smaller'} than L2",
                "parallelism": f"independent trees per GPU x{world}"}

    def setup(self, rank, dev):
        import gen.basis_tree as gb
        import paper_1707_05141_gb300 as bs
        self.bs = bs
        self.tree = gb.chebyshev_basis_tree(self.depth, q=8, seed_index=rank)
        self.plan = bs.H2Plan(self.tree.leaves, self.tree.transfers, self.tree.k)
        self.d_in = [self.plan.leaf, self.plan.E]
        self.h_in = None
        self.outs = [self.plan.new_leaf, self.plan.new_transfer, self.plan.T, self.plan.rank]
        self.launches_per_step = 1 + 2 + 3 * self.depth   # setup, leaves (SVD, finish), per level (TE, SVD, finish)

    def step(self, stream, kev=None):
        if kev is not None:
            kev[0].record(stream)
        self.plan.run(1e-5, stream)
        if kev is not None:
            kev[1].record(stream)

    def roofline(self, kernel_ms):
        p = self.plan
        info = p.info.cpu().numpy()
        rot = p.rotations.cpu().numpy().astype(np.float64)
        rank = p.rank.cpu().numpy()
        nl = 2 ** self.depth
        k = p.k
        sweeps = np.where(info >= (1 << 20), info - (1 << 20), np.maximum(info, 0)).astype(np.float64)
        # Jacobi flops per node: pairs visited 6 max(m, n) per sweep, rotations 6 (m + n)
        rows = np.empty(2 * nl - 1)
        rows[nl - 1:] = p.m
        for g in range(nl - 2, -1, -1):
            rows[g] = rank[2 * g + 1] + rank[2 * g + 2]
        kmin = np.minimum(rows, k)
        fl = float(np.sum(sweeps * kmin * (kmin - 1) / 2 * 6 * np.maximum(rows, k) + rot * 6 * (rows + k)))
        achieved = fl / (kernel_ms * 1e-3) / 1e12
        return ({"kernel": "bsvd_h2_truncate (all levels of one tree)", "bound": "alu", "achieved": achieved,
                 "peak": PEAKS["fp32"]["tflops"], "unit": "TFLOP/s", "frac": achieved / PEAKS["fp32"]["tflops"],
                 "traffic": None, "ms_per_launch": kernel_ms,
                 "peak_note": PEAKS["fp32"]["note"] + "; achieved counts the Jacobi flops of every node's SVD"},
                {"leaves_per_s": nl / (kernel_ms * 1e-3), "leaf_rank_mean": float(rank[nl - 1:].mean()),
                 "root_rank": int(rank[0]), "sweeps_mean_leaves": float(sweeps[nl - 1:].mean())})

    def cpu_sample(self, n):
        import oracle.h2 as oh2
        import gen.basis_tree as gb
        import oracle
        d = 6
        tree = gb.chebyshev_basis_tree(d, q=8)
        t0 = time.time()
        oh2.truncate_basis_tree(tree.leaves, tree.transfers, 1e-5)
        dt = time.time() - t0
        # per-leaf rate of a depth-6 tree, scaled to the benchmark's tree (leaves dominate the work)
        per_tree = dt * (2 ** self.depth) / (2 ** d)
        return {"value": 1.0 / per_tree, "count": 1, "seconds": per_tree, "unit": self.unit, "cores": 1,
                "kind": "oracle", "sample": f"one depth-{d} tree ({2 ** d} leaves) by the FP64 oracle in {dt:.2f} s "
                                            f"(one thread), scaled by leaf count to depth {self.depth}"}


WORKLOADS = {c.name: c for c in (SvdQr64, Fp64_32, Block512, RsvdUneven, HmatrixMlp, H2Truncation)}


# ----------------------------------------------------------------------------------------------
# harness
# ----------------------------------------------------------------------------------------------

def time_arm(step, stream, steps, local_rank, world, dev, flush=None, profile=False):
    """Times exactly `steps` calls of step(stream, events) on `stream` with CUDA events, between a
    barrier and a synchronize on both sides, with the SM clocks sampled meanwhile.  With `flush` (a
    buffer larger than L2) L2 is overwritten before every step, outside that step's own events.
    With `profile` the region is bracketed by cudaProfilerStart/Stop, so that a profiler started
    with profiling off (ncu --profile-from-start off) records exactly the timed steps.
    Returns the per-step time (max over ranks), the mean time between the events the step records
    around its dominant call, and the clock record."""
    import torch
    kev, step_ev = [], []
    clocks = Clocks(local_rank)
    clocks.start()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    if profile:
        torch.cuda.profiler.start()
    t0e, t1e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    wall0 = time.time()
    t0e.record(stream)
    for _ in range(steps):
        ev = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
        if flush is not None:
            flush.fill_(1)
            se = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
            se[0].record(stream)
        step(stream, ev)
        if flush is not None:
            se[1].record(stream)
            step_ev.append(se)
        kev.append(ev)
    t1e.record(stream)
    torch.cuda.synchronize()
    if profile:
        torch.cuda.profiler.stop()
    wall1 = time.time()
    if world > 1:
        torch.distributed.barrier()
    ck = clocks.stop(wall0, wall1)
    own_ms = (sum(a.elapsed_time(b) for a, b in step_ev) if step_ev else t0e.elapsed_time(t1e)) / steps
    return {"ms_step": max_over_ranks(own_ms, world, dev),
            "kernel_ms": statistics.mean(a.elapsed_time(b) for a, b in kev), "clocks": ck}


def run_ours(W, args, rank, world, local_rank):
    import torch
    import paper_1707_05141_gb300 as bs

    bs.lib()  # fail loudly when the library is missing
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    W.setup(rank, dev)
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        W.step(stream)
    torch.cuda.synchronize()
    if hasattr(W, "capture"):
        W.capture(stream)
        W.step(stream)
        torch.cuda.synchronize()
    # a batch smaller than L2 is evicted before every timed step by writing a buffer larger than L2
    # (256 MB against 129 MB); each step then has its own events, which exclude the flush
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev) if getattr(W, "flush_l2", False) else None
    t = time_arm(W.step, stream, args.steps, local_rank, world, dev, flush, profile=args.profile_timed)
    ms_step, kernel_ms, ck = t["ms_step"], t["kernel_ms"], t["clocks"]
    roof, detail = W.roofline(kernel_ms)

    # the plain form of the same workload (FP32 SIMT products, no learned or given ranks), timed
    # the same way over the same number of steps: the "mixed vs plain FP32 at 1e-5" comparison
    if hasattr(W, "plain_arm"):
        quality = W.quality()
        pstep, pfinish = W.plain_arm(stream)
        for _ in range(args.warmup):
            pstep(stream)
        torch.cuda.synchronize()
        pt = time_arm(pstep, stream, args.steps, local_rank, world, dev, flush)
        detail["mixed_vs_plain"] = {
            "mixed": {"form": W.mixed_form, "ms_per_step": ms_step, "clocks": ck, **quality},
            "plain": {"form": W.plain_form, "ms_per_step": pt["ms_step"], "clocks": pt["clocks"], **pfinish()},
            "speedup": pt["ms_step"] / ms_step}
    if hasattr(W, "extra_arms"):
        # the other forms of the workload (reported beside the timed one): fewer steps each
        xs = max(1, min(args.steps, 5))
        extra = W.extra_arms(stream, xs, args.warmup,
                             lambda step: dict(time_arm(step, stream, xs, local_rank, world, dev, flush), steps=xs))
        detail.update(extra)
    if hasattr(W, "train_info"):
        detail["training"] = W.train_info

    # end to end through the public API: pinned host inputs copied in, every output copied out.
    # Workloads with a host entry (uniform SVD + QR batches) call the library's host-in/host-out
    # functions, whose chunked copies overlap the computation (bsvd_host_qr / bsvd_host_svd); the
    # others copy with torch around their device call.
    if getattr(W, "h_in", None) is None:
        W.h_in = [d.cpu().pin_memory() for d in W.d_in]
    houts = [torch.empty(o.shape, dtype=o.dtype).pin_memory() for o in W.outs]
    e2e_steps = max(1, min(args.steps, 5))
    host_step = W.host_step(houts, args.e2e_chunks) if hasattr(W, "host_step") else None

    def e2e_step():
        if host_step is not None:
            host_step(stream)
            return
        for d, h in zip(W.d_in, W.h_in):
            d.copy_(h, non_blocking=True)
        W.step(stream)
        for h, o in zip(houts, W.outs):
            h.copy_(o, non_blocking=True)

    e2e_step()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    x0, x1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    x0.record(stream)
    for _ in range(e2e_steps):
        e2e_step()
    x1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks(x0.elapsed_time(x1) / e2e_steps, world, dev)
    h2d = sum(h.numel() * h.element_size() for h in W.h_in)
    d2h = sum(h.numel() * h.element_size() for h in houts)
    return {"ms_step": ms_step, "value": world * W.units / (ms_step * 1e-3),
            "e2e": {"value": world * W.units / (e2e_ms * 1e-3), "unit": W.unit, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms,
                    "path": ("C ABI host entries (bsvd_host_qr, bsvd_host_svd), "
                             f"{args.e2e_chunks} overlapped chunks") if host_step is not None
                    else "torch copies around the device entry points, serial"},
            "roofline": roof, "clocks": ck, "gpu_launches": W.launches_per_step * args.steps, "detail": detail}


SECONDARY = ("fp64_32", "block512", "rsvd_uneven", "hmatrix_mlp", "h2_truncation")
CPU_SAMPLE = {"svd64_qr128": 4000, "fp64_32": 1000, "block512": 4, "rsvd_uneven": 256, "hmatrix_mlp": 512,
              "h2_truncation": 1}
# bounded oracle samples of the other workloads in a default run (a few seconds of host time each)
CPU_SAMPLE_SECONDARY = {"fp64_32": 500, "block512": 2, "rsvd_uneven": 96, "hmatrix_mlp": 256, "h2_truncation": 1}


def line_of(W, res, args, world, cb):
    return {"metric": W.metric, "value": res["value"], "unit": W.unit, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": res["ms_step"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": W.dtype, "data": "synthetic", "config": W.config(world),
            "roofline": res["roofline"], "cpu_baseline": cb, "e2e": res["e2e"], "clocks": res["clocks"],
            "gpu_launches": res["gpu_launches"], "detail": res["detail"]}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default=None,
                    help="time this workload alone (default: svd64_qr128 as the headline line, the other four "
                         "in detail.workloads)")
    ap.add_argument("--headline-only", action="store_true", help="default run without the other workloads")
    ap.add_argument("--host-inputs", action="store_true",
                    help="block512 / rsvd_uneven inputs from the host generator (byte-identical to the tests', "
                         "minutes of LAPACK time) instead of the same recipe on the device")
    ap.add_argument("--svd-batch", type=int, default=20000)
    ap.add_argument("--jacobi-tier", default=None,
                    help="svd64_qr128: run this encoded register variant (e.g. 0xa01) instead of autotuning")
    ap.add_argument("--qr-batch", type=int, default=20000)
    ap.add_argument("--block-batch", type=int, default=500, help="block512: matrices per GPU")
    ap.add_argument("--rsvd-batch", type=int, default=16384, help="rsvd_uneven: blocks per GPU")
    ap.add_argument("--e2e-chunks", type=int, default=8,
                    help="chunks of the host entries' end-to-end run whose copies overlap the computation")
    ap.add_argument("--cpu-sample", type=int, default=0, help="oracle sample size (0: per-workload default)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--profile-timed", action="store_true",
                    help="bracket the main timed steps by cudaProfilerStart/Stop (ncu --profile-from-start off)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    name = args.workload or "svd64_qr128"
    W = WORKLOADS[name](args)
    ns = args.cpu_sample or CPU_SAMPLE[W.name]

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        # the reference arm is the FP64 oracle on the host cores (the paper ships no code)
        if rank != 0:
            return
        # W untimed warm-up samples, then K timed ones; each step a bounded sample (the default
        # sample split over the K steps), the value total units / total oracle time
        k = max(1, args.steps)
        per = max(1, ns // k)
        for _ in range(args.warmup):
            W.cpu_sample(per)
        vals = [W.cpu_sample(per) for _ in range(k)]
        count = sum(x["count"] for x in vals)
        seconds = sum(x["seconds"] for x in vals)
        v = count / seconds
        cb = {key: val for key, val in vals[0].items() if key not in ("count", "seconds")}
        cb["value"] = v
        cb["sample"] = f"{k} steps of {per}: " + cb["sample"]
        print(json.dumps({"impl": "reference", "metric": W.metric, "value": v, "unit": W.unit, "n_gpus": world,
                          "steps": k, "warmup": args.warmup, "ms_per_step": 1e3 * seconds / k,
                          "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                          "data": "synthetic", "config": W.config(world), "cpu_baseline": cb,
                          "e2e": {"value": v, "unit": W.unit, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))
        return

    import torch
    if world > 1:
        torch.distributed.init_process_group("nccl")
    import paper_1707_05141_gb300 as bs
    torch.cuda.set_device(torch.device("cuda", local_rank))
    measure_alu_peaks(bs, torch.device("cuda", local_rank), local_rank)
    res = run_ours(W, args, rank, world, local_rank)
    cb = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cb = {key: val for key, val in W.cpu_sample(ns).items() if key not in ("count", "seconds")}
    line = line_of(W, res, args, world, cb)
    line["detail"]["alu_peaks"] = PEAKS
    if args.workload is None and not args.headline_only:
        # the other four workloads, each timed the same way (K steps after W warm-ups, clocks,
        # roofline, plain arm, end to end, bounded oracle sample), one after the other
        del W
        torch.cuda.empty_cache()
        others = {}
        for other in SECONDARY:
            W2 = WORKLOADS[other](args)
            r2 = run_ours(W2, args, rank, world, local_rank)
            cb2 = None
            if rank == 0 and world == 1 and not args.no_cpu_baseline:
                cb2 = {key: val for key, val in W2.cpu_sample(CPU_SAMPLE_SECONDARY[other]).items()
                       if key not in ("count", "seconds")}
            l2 = line_of(W2, r2, args, world, cb2)
            others[other] = {k: v for k, v in l2.items() if k not in ("n_gpus", "scaling", "vs_baseline", "data",
                                                                       "higher_is_better", "warmup")}
            del W2
            torch.cuda.empty_cache()
        line["detail"]["workloads"] = others
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
