#!/usr/bin/env python
"""Benchmark of the batched Jacobi SVD / Householder QR path on one GB300 (or N, weak scaling).

Default workload ("svd64_qr128"): one step = batched Householder QR of 20000 FP32 128 x 32
matrices + batched one-sided Jacobi SVD (U, S, V) of 20000 FP32 64 x 64 matrices, the matrices
built as U diag(sigma) V^T with Haar U, V and sigma_i = exp(-i/8).  The metric is SVDs per second
(whole job); inputs are resident in HBM (656 MB, larger than the 129 MB L2) when the timed region
starts.  Also reported: the dominant kernel against its roofline, an end-to-end figure through
the public API with host buffers, and the FP64 oracle on the host cores as the CPU baseline.

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

# FP32 SIMT peak: 152 SMs x 128 FP32 lanes x 2 flops (FMA) x 2.070 GHz maximum SM clock
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12
# FP64 peak of the part (GB300 data sheet figure, for the FP64 workload only)
FP64_PEAK_TFLOPS = 1.25

# DRAM bytes (read + write) per launch of the dominant kernel from one ncu capture, valid only for
# the kernel source it was taken on (the digest guards against reporting stale counters).
TRAFFIC = {}


def kernel_digest(name: str) -> str:
    p = os.path.join(ROOT, "paper_1707_05141_gb300", "csrc", name)
    with open(p, "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()[:16]


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


# ----------------------------------------------------------------------------------------------
# workload
# ----------------------------------------------------------------------------------------------

def jacobi_flops(m, n, info, rots):
    """Algorithmic flops of one-sided Jacobi: every visited pair costs its 2x2 Gram (6m), every
    applied rotation 6(m + n) (A and V columns); sweeps = info (or info - NOT_CONVERGED)."""
    sweeps = np.where(info >= (1 << 20), info - (1 << 20), info).astype(np.float64)
    k = min(m, n)
    mm = max(m, n)
    return float(np.sum(sweeps * (k * (k - 1) / 2) * 6 * mm + rots.astype(np.float64) * 6 * (m + n)))


def qr_flops(m, n):
    return 4.0 * m * n * n - 4.0 * n ** 3 / 3.0 + 4.0 * m * n * n - 4.0 * n ** 3 / 3.0  # factor + form Q


def make_inputs(rank: int, svd_batch: int, qr_batch: int):
    import gen
    a_svd = gen.workload1_svd(batch=svd_batch, first=rank * svd_batch)
    a_qr = gen.workload1_qr(batch=qr_batch, first=rank * qr_batch)
    return a_svd, a_qr


def run_ours(args, rank, world, local_rank):
    import torch
    import paper_1707_05141_gb300 as bs

    bs.lib()  # fail loudly when the library is missing
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    nb_svd, nb_qr = args.svd_batch, args.qr_batch
    a_svd, a_qr = make_inputs(rank, nb_svd, nb_qr)
    h_svd = torch.from_numpy(a_svd.a).pin_memory()
    h_qr = torch.from_numpy(a_qr.a).pin_memory()
    d_svd = h_svd.to(dev)
    d_qr = h_qr.to(dev)
    m, n = 64, 64
    mq, nq = 128, 32
    k = 64
    A = bs.Batch.uniform(d_svd, m, n)
    S = torch.empty((nb_svd, 1, k), device=dev)
    U = torch.empty((nb_svd, k, m), device=dev)
    V = torch.empty((nb_svd, k, n), device=dev)
    Sb, Ub, Vb = bs.Batch.uniform(S, k, 1), bs.Batch.uniform(U, m, k), bs.Batch.uniform(V, n, k)
    info = torch.empty(nb_svd, dtype=torch.int32, device=dev)
    rots = torch.empty(nb_svd, dtype=torch.int64, device=dev)
    AQ = bs.Batch.uniform(d_qr, mq, nq)
    Q = torch.empty((nb_qr, nq, mq), device=dev)
    R = torch.empty((nb_qr, nq, nq), device=dev)
    Qb, Rb = bs.Batch.uniform(Q, mq, nq), bs.Batch.uniform(R, nq, nq)
    qinfo = torch.empty(nb_qr, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream()
    from paper_1707_05141_gb300 import autotune
    tuned = autotune.tune_jacobi(d_svd, m, n)   # picks tier/variant for this size bin (not timed)

    ev = []

    def step(record=False):
        bs.batched_qr(AQ, Qb, Rb, qinfo, stream)
        if record:
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
        bs.batched_svd_jacobi(A, Sb, Ub, Vb, info, rots, stream=stream)
        if record:
            e1.record(stream)
            ev.append((e0, e1))

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    clocks = Clocks(local_rank)
    clocks.start()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    wall0 = time.time()
    t_start.record(stream)
    for _ in range(args.steps):
        step(record=True)
    t_end.record(stream)
    torch.cuda.synchronize()
    wall1 = time.time()
    if world > 1:
        torch.distributed.barrier()
    ck = clocks.stop(wall0, wall1)
    ms_total = t_start.elapsed_time(t_end)
    jac_ms = statistics.mean(e0.elapsed_time(e1) for e0, e1 in ev)
    if world > 1:
        t = torch.tensor([ms_total], device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms_total = float(t.item())
    ms_step = ms_total / args.steps

    info_h = info.cpu().numpy()
    rots_h = rots.cpu().numpy()
    assert np.all(info_h > 0), "Jacobi reported a bad shape"
    fl = jacobi_flops(m, n, info_h, rots_h)
    achieved = fl / (jac_ms * 1e-3) / 1e12
    tier = int(tuned["tier"])
    kname = ("jacobi_reg_kernel" if (tier & 0xff) == bs.TIER_REGISTER else "jacobi_smem_kernel") + f" (tier {tier:#x})"
    dig = kernel_digest("jacobi_reg.cu" if (tier & 0xff) == bs.TIER_REGISTER else "jacobi_smem.cu")
    traffic = TRAFFIC.get(dig)

    # ---- end to end through the public API: pinned host in, host out ----
    o_s = torch.empty((nb_svd, 1, k)).pin_memory()
    o_u = torch.empty((nb_svd, k, m)).pin_memory()
    o_v = torch.empty((nb_svd, k, n)).pin_memory()
    o_q = torch.empty((nb_qr, nq, mq)).pin_memory()
    o_r = torch.empty((nb_qr, nq, nq)).pin_memory()
    e2e_steps = max(1, min(args.steps, 10))

    def e2e_step():
        d_svd.copy_(h_svd, non_blocking=True)
        d_qr.copy_(h_qr, non_blocking=True)
        step()
        o_s.copy_(S, non_blocking=True)
        o_u.copy_(U, non_blocking=True)
        o_v.copy_(V, non_blocking=True)
        o_q.copy_(Q, non_blocking=True)
        o_r.copy_(R, non_blocking=True)

    e2e_step()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    x0 = torch.cuda.Event(enable_timing=True)
    x1 = torch.cuda.Event(enable_timing=True)
    x0.record(stream)
    for _ in range(e2e_steps):
        e2e_step()
    x1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = x0.elapsed_time(x1) / e2e_steps
    if world > 1:
        t = torch.tensor([e2e_ms], device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        e2e_ms = float(t.item())
    h2d = h_svd.numel() * 4 + h_qr.numel() * 4
    d2h = sum(t.numel() * 4 for t in (o_s, o_u, o_v, o_q, o_r))

    return {
        "ms_step": ms_step,
        "value": world * nb_svd / (ms_step * 1e-3),
        "e2e": {"value": world * nb_svd / (e2e_ms * 1e-3), "unit": "SVDs/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms},
        "roofline": {"kernel": kname, "bound": "alu", "achieved": achieved,
                     "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": achieved / FP32_PEAK_TFLOPS,
                     "traffic": traffic, "ms_per_launch": jac_ms,
                     "peak_note": "FP32 SIMT: 152 SMs x 128 lanes x 2 flops x 2.07 GHz (max SM clock)"},
        "clocks": ck,
        "gpu_launches": 2 * args.steps,
        "detail": {"svd_sweeps_mean": float(np.mean(info_h)), "rotations_mean": float(np.mean(rots_h)),
                   "jacobi_gflop_per_launch": fl / 1e9, "autotune": tuned},
    }


def cpu_baseline(args, n_svd, n_qr):
    """The FP64 oracle (as it stands) on a bounded sample of the same workload, all host cores."""
    import oracle
    a_svd, a_qr = make_inputs(0, n_svd, n_qr)
    mats = [a_svd.a64(i) for i in range(n_svd)]
    qmats = [a_qr.a64(i) for i in range(n_qr)]
    cores = oracle.default_threads()
    t0 = time.time()
    oracle.svd_batch(mats, tol=-1.0, nthreads=cores)
    oracle.qr_batch(qmats, nthreads=cores)
    dt = time.time() - t0
    # one step's unit of work is (1 SVD of 64x64 + 1 QR of 128x32) per SVD counted
    return {"value": n_svd / dt, "unit": "SVDs/s", "cores": cores, "kind": "oracle",
            "sample": f"{n_svd} SVDs of 64x64 + {n_qr} QRs of 128x32 (same generator), FP64, {dt:.2f} s wall"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=60)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--svd-batch", type=int, default=20000)
    ap.add_argument("--qr-batch", type=int, default=20000)
    ap.add_argument("--cpu-sample", type=int, default=4000)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    config = {"workload": "svd64_qr128: Jacobi SVD (U,S,V) of 20000 FP32 64x64 + Householder QR (Q,R) of 20000 "
                          "FP32 128x32 per GPU per step; sigma_i = exp(-i/8), Haar U, V",
              "svd_batch_per_gpu": args.svd_batch, "qr_batch_per_gpu": args.qr_batch, "m": 64, "n": 64,
              "qr_m": 128, "qr_n": 32, "l2": "inputs (656 MB per GPU) larger than L2; no flush",
              "parallelism": f"independent batches per GPU x{world}"}
    metric = "batched SVDs/s (64x64 FP32 Jacobi SVD + 128x32 FP32 QR per SVD)"

    if args.impl == "reference":
        if rank != 0:
            return
        vals = []
        n = max(1, args.cpu_sample // 4)
        for _ in range(args.warmup if args.warmup < 1 else 1):
            cpu_baseline(args, 64, 64)
        for _ in range(args.steps if args.steps <= 5 else 5):
            vals.append(cpu_baseline(args, n, n))
        v = statistics.median(x["value"] for x in vals)
        cb = dict(vals[0])
        cb["value"] = v
        print(json.dumps({"impl": "reference", "metric": metric, "value": v, "unit": "SVDs/s", "n_gpus": 0,
                          "steps": len(vals), "warmup": args.warmup, "ms_per_step": 1e3 * args.svd_batch / v,
                          "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                          "data": "synthetic", "config": config, "cpu_baseline": cb,
                          "e2e": {"value": v, "unit": "SVDs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))
        return

    if world > 1:
        import torch
        torch.distributed.init_process_group("nccl")
    res = run_ours(args, rank, world, local_rank)
    cb = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cb = cpu_baseline(args, args.cpu_sample, args.cpu_sample)
    if rank == 0:
        line = {"metric": metric, "value": res["value"], "unit": "SVDs/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": res["ms_step"], "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": config,
                "roofline": res["roofline"], "cpu_baseline": cb, "e2e": res["e2e"], "clocks": res["clocks"],
                "gpu_launches": res["gpu_launches"], "detail": res["detail"]}
        print(json.dumps(line))
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
