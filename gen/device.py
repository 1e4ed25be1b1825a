"""Device-side generation of the two largest benchmark inputs (the 500 x 512^2 batch and the 16 384
uneven blocks), by the host generator's recipe: A = U diag(sigma) V^T with Haar U, V (QR of a
Gaussian matrix, columns multiplied by sign(diag R)), formed in FP64 and rounded to FP32.

The host generator needs minutes of LAPACK time for these batches; here the Gaussian entries come
from torch's Philox generator on the GPU (seeded from the base seed, the workload and the first
matrix index) and the QR and products run on the device.  The bytes therefore differ from the host
generator's, while the spectra (and, for the uneven blocks, the shapes and decay rates) are drawn
from the host generator's own streams, so the workloads are the same in distribution.  Like the host
generator, this module holds none of the method's arithmetic: the QR is a library primitive used
only to sample the orthogonal group.
"""
from __future__ import annotations

import math

import numpy as np

from . import BASE_SEED, TAG_SHAPE, sigma_decay, sigma_loguniform, uniforms


def _torch():
    import torch
    return torch


def _generator(dev, workload: int, first: int):
    torch = _torch()
    g = torch.Generator(device=dev)
    g.manual_seed((BASE_SEED * 1000003 + workload * 7919 + first) & 0x7FFFFFFFFFFFFFFF)
    return g


def _haar(cnt: int, rows: int, cols: int, dev, g):
    """cnt Haar-distributed rows x cols orthonormal factors (FP64, device)."""
    torch = _torch()
    z = torch.randn((cnt, rows, cols), generator=g, device=dev, dtype=torch.float64)
    q, r = torch.linalg.qr(z)
    d = torch.sign(torch.diagonal(r, dim1=-2, dim2=-1))
    d[d == 0] = 1.0
    return q * d[:, None, :]


def block512_loguniform(batch: int = 500, first: int = 0, size: int = 512, dev="cuda", chunk: int = 64):
    """(a, sigma): a of shape (batch, size, size) FP32 on ``dev`` (matrix b is a[b].T), sigma (batch, size)
    log-uniform on [1e-6, 1] from the host generator's sigma stream of workload 2."""
    torch = _torch()
    g = _generator(dev, 2, first)
    a = torch.empty((batch, size, size), device=dev, dtype=torch.float32)
    sig = np.stack([sigma_loguniform(2, i, size) for i in range(first, first + batch)])
    for c0 in range(0, batch, chunk):
        c1 = min(batch, c0 + chunk)
        u = _haar(c1 - c0, size, size, dev, g)
        v = _haar(c1 - c0, size, size, dev, g)
        s = torch.as_tensor(sig[c0:c1], device=dev)
        m = torch.bmm(u * s[:, None, :], v.transpose(1, 2))
        a[c0:c1] = m.transpose(1, 2).to(torch.float32)
    return a, sig


def rsvd_uneven_blocks(batch: int = 16384, first: int = 0, sizes=(64, 128, 256), eps: float = 1e-5, dev="cuda",
                       chunk: int = 512):
    """(flat, offset, m, n, r0, rank_hint): the uneven workload packed in one FP32 device tensor
    (column-major blocks at element ``offset``, 4-element aligned); shapes and r0 from the host
    generator's shape stream of workload 3, sigma_i = exp(-i / r0)."""
    torch = _torch()
    sizes = np.asarray(sizes)
    ms, ns, r0s = [], [], []
    for i in range(first, first + batch):
        u = uniforms(3, i, TAG_SHAPE, 3)
        ms.append(int(sizes[min(int(u[0] * len(sizes)), len(sizes) - 1)]))
        ns.append(int(sizes[min(int(u[1] * len(sizes)), len(sizes) - 1)]))
        r0s.append(2.0 + 10.0 * u[2])
    ms = np.array(ms, np.int32)
    ns = np.array(ns, np.int32)
    r0s = np.array(r0s)
    padded = (ms.astype(np.int64) * ns + 3) // 4 * 4
    off = np.zeros(batch, np.int64)
    off[1:] = np.cumsum(padded)[:-1]
    flat = torch.zeros(int(padded.sum()), device=dev, dtype=torch.float32)
    g = _generator(dev, 3, first)
    for mm in sizes:
        for nn in sizes:
            idx = np.nonzero((ms == mm) & (ns == nn))[0]
            k = int(min(mm, nn))
            for c0 in range(0, len(idx), chunk):
                sel = idx[c0:c0 + chunk]
                u = _haar(len(sel), int(mm), k, dev, g)
                v = _haar(len(sel), int(nn), k, dev, g)
                s = torch.as_tensor(np.stack([sigma_decay(r0s[b], k) for b in sel]), device=dev)
                a = torch.bmm(u * s[:, None, :], v.transpose(1, 2)).transpose(1, 2).reshape(len(sel), -1)
                a = a.to(torch.float32)
                # scatter the column-major blocks to their offsets
                pos = torch.as_tensor(off[sel], device=dev)[:, None] + torch.arange(int(mm) * int(nn), device=dev)
                flat[pos.reshape(-1)] = a.reshape(-1)
    hint = np.minimum(np.ceil(r0s * math.log(1.0 / eps)).astype(np.int32), np.minimum(ms, ns))
    return flat, off, ms, ns, r0s, hint
