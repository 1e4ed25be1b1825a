"""Autotuner for the Jacobi SVD tiers.

For one size bin (dtype, max(m, n), min(m, n)) it times every kernel variant that can run the
batch -- the register-tier variants (pair slots, row parts per matrix, resident CTAs per SM,
scaled or plain rotations) and the shared-memory tier -- on a sample of the caller's batch,
records the fastest with ``bsvd_set_jacobi_choice`` so that ``TIER_AUTO`` uses it, and caches
the choice per GPU model in ``_build/autotune.json``.  For the block tier it times the block
widths (16, 32) and, for GRAM, the inner register variant of the pair SVDs, and records the fastest
with ``bsvd_set_block_choice`` (``block_width = 0`` uses it).  The paper tunes its kernels by hand
for one GPU (panel width, matrices per block, block width, Sections 3-6); this replaces that with
measurement.
"""
from __future__ import annotations

import json
import os
import threading

from . import (BLOCK_GRAM, F32, F64, LIB, TIER_REGISTER, TIER_SHARED, Batch, batched_svd_block_jacobi,
               batched_svd_block_jacobi_workspace, batched_svd_jacobi, jacobi_variant_desc, jacobi_variants,
               set_block_choice, set_jacobi_choice)

CACHE = os.path.join(os.path.dirname(LIB), "autotune.json")
_lock = threading.Lock()


def _bin(x: int) -> int:
    b = 0
    while (1 << b) < x and b < 8:
        b += 1
    return b


def _key(gpu: str, code: int, m: int, n: int) -> str:
    mm, nn = max(m, n), min(m, n)
    return f"{gpu}|{'f32' if code == F32 else 'f64'}|{_bin(mm)}|{_bin(nn)}"


def _load():
    try:
        with open(CACHE) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(d):
    tmp = CACHE + f".{os.getpid()}.tmp"
    with open(tmp, "w") as f:
        json.dump(d, f, indent=1, sort_keys=True)
    os.replace(tmp, CACHE)


def candidates(code: int, m: int, n: int):
    tiers = [TIER_REGISTER | (v << 8) for v in range(1, jacobi_variants(code, m, n, TIER_REGISTER) + 1)]
    if jacobi_variants(code, m, n, TIER_SHARED) > 0:
        tiers.append(TIER_SHARED)
    return tiers


def tune_jacobi(a, m: int | None = None, n: int | None = None, sample: int = 3648, reps: int = 2,
                want_vectors: bool = True, force: bool = False) -> dict:
    """Tune the size bin of the uniform batch ``a`` (batch, n, m) on its device; returns the record."""
    import torch

    bsz, cols, ld = a.shape
    m = ld if m is None else m
    n = cols if n is None else n
    code = F32 if a.dtype == torch.float32 else F64
    gpu = torch.cuda.get_device_name(a.device)
    key = _key(gpu, code, m, n)
    with _lock:
        cache = _load()
        if key in cache and not force:
            rec = cache[key]
            set_jacobi_choice(code, m, n, int(rec["tier"]))
            return rec
    s = a[: min(bsz, sample)].contiguous()
    nb = s.shape[0]
    k = min(m, n)
    A = Batch.uniform(s, m, n)
    S = torch.empty((nb, 1, k), device=a.device, dtype=a.dtype)
    U = torch.empty((nb, k, m), device=a.device, dtype=a.dtype) if want_vectors else None
    V = torch.empty((nb, k, n), device=a.device, dtype=a.dtype) if want_vectors else None
    info = torch.empty(nb, device=a.device, dtype=torch.int32)
    Sb = Batch.uniform(S, k, 1)
    Ub = Batch.uniform(U, m, k) if want_vectors else None
    Vb = Batch.uniform(V, n, k) if want_vectors else None
    times = {}
    for t in candidates(code, m, n):
        batched_svd_jacobi(A, Sb, Ub, Vb, info, tier=t)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            batched_svd_jacobi(A, Sb, Ub, Vb, info, tier=t)
        e1.record()
        torch.cuda.synchronize()
        times[t] = e0.elapsed_time(e1) / reps
    best = min(times, key=times.get)
    set_jacobi_choice(code, m, n, best)
    rec = {"tier": best, "ms": times[best], "sample": nb, "all_ms": {hex(t): v for t, v in times.items()}}
    with _lock:
        cache = _load()
        cache[key] = rec
        _store(cache)
    return rec


def apply_cache(device=None) -> int:
    """Re-apply every cached choice for this GPU model; returns how many were applied."""
    import torch

    gpu = torch.cuda.get_device_name(device)
    n = 0
    for key, rec in _load().items():
        parts = key.split("|")
        if parts[0] == "block":
            _, g, dt, bm, bn, _m = parts
            if g == gpu:
                set_block_choice(F32 if dt == "f32" else F64, 1 << int(bm), 1 << int(bn), int(rec["block_width"]),
                                 int(rec["inner_variant"]))
                n += 1
            continue
        g, dt, bm, bn = parts
        if g != gpu:
            continue
        set_jacobi_choice(F32 if dt == "f32" else F64, 1 << int(bm), 1 << int(bn), int(rec["tier"]))
        n += 1
    return n


def _block_bin(x: int) -> int:
    b = 0
    while (1 << b) < x and b < 14:
        b += 1
    return b


def _block_key(gpu: str, code: int, m: int, n: int, method: int) -> str:
    mm, nn = max(m, n), min(m, n)
    return f"block|{gpu}|{'f32' if code == F32 else 'f64'}|{_block_bin(mm)}|{_block_bin(nn)}|{method & 0xff}"


def block_candidates(code: int, method: int):
    """(block width, inner variant) pairs: both widths with the default inner SVD and, for GRAM, the
    register variants with carried column norms for the 2bw x 2bw Gram matrices, QR-preconditioned
    (X = its U) and plain (X = its V, no QR of G: cheaper per visit, fewer sweeps' worth of
    progress in the capped inner SVD)."""
    out = []
    for bw in (16, 32):
        out.append((bw, 0))
        if (method & 0xff) == BLOCK_GRAM:
            k2 = 2 * bw
            nv = jacobi_variants(code, k2, k2, TIER_REGISTER)
            for pre in (1, 0):
                for k in range(1, nv + 1):
                    d = jacobi_variant_desc(code, k2, k2, k)
                    if d["qr_precond"] == pre and d["carried_norms"]:
                        out.append((bw, k))
                        break
    return out


def tune_block(a, method: int = BLOCK_GRAM, m: int | None = None, n: int | None = None, sample: int = 64,
               reps: int = 1, force: bool = False) -> dict:
    """Tune the block tier's width and inner variant for the size bin of the uniform batch ``a``
    (batch, n, m) and ``method`` (its flag bits included in the timing); returns the record."""
    import torch

    bsz, cols, ld = a.shape
    m = ld if m is None else m
    n = cols if n is None else n
    code = F32 if a.dtype == torch.float32 else F64
    gpu = torch.cuda.get_device_name(a.device)
    key = _block_key(gpu, code, m, n, method)
    with _lock:
        cache = _load()
        if key in cache and not force:
            rec = cache[key]
            set_block_choice(code, m, n, int(rec["block_width"]), int(rec["inner_variant"]))
            return rec
    s = a[: min(bsz, sample)].contiguous()
    nb = s.shape[0]
    k = min(m, n)
    A = Batch.uniform(s, m, n)
    S = torch.empty((nb, 1, k), device=a.device, dtype=a.dtype)
    U = torch.empty((nb, k, m), device=a.device, dtype=a.dtype)
    V = torch.empty((nb, k, n), device=a.device, dtype=a.dtype)
    info = torch.empty(nb, device=a.device, dtype=torch.int32)
    Sb, Ub, Vb = Batch.uniform(S, k, 1), Batch.uniform(U, m, k), Batch.uniform(V, n, k)
    times = {}
    for bw, inner in block_candidates(code, method):
        meth = method | (inner << 8)
        ws = torch.empty(max(batched_svd_block_jacobi_workspace(A, bw, meth), 1), dtype=torch.uint8,
                         device=a.device)
        batched_svd_block_jacobi(A, Sb, Ub, Vb, info, ws, block_width=bw, method=meth)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            batched_svd_block_jacobi(A, Sb, Ub, Vb, info, ws, block_width=bw, method=meth)
        e1.record()
        torch.cuda.synchronize()
        times[(bw, inner)] = e0.elapsed_time(e1) / reps
        del ws
    bw, inner = min(times, key=times.get)
    set_block_choice(code, m, n, bw, inner)
    rec = {"block_width": bw, "inner_variant": inner, "ms": times[(bw, inner)], "sample": nb,
           "all_ms": {f"bw{b}_inner{i}": v for (b, i), v in times.items()}}
    with _lock:
        cache = _load()
        cache[key] = rec
        _store(cache)
    return rec
