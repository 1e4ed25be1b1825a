"""Seeded synthetic inputs for the batched QR / Jacobi SVD / randomized SVD workloads.

This module only *makes test matrices*; it holds none of the method's arithmetic.  Both the
FP64 oracle (``oracle/``) and the CUDA library are fed from here, and neither is imported.

Every matrix is ``A = U diag(sigma) V^T`` with Haar-distributed orthonormal ``U`` (m x k) and
``V`` (n x k), k = min(m, n).  Haar factors are drawn the standard way (Mezzadri 2007): QR of a
Gaussian matrix by LAPACK (``numpy.linalg.qr``, a library primitive used only to sample the
orthogonal group) followed by multiplying column j by sign(R_jj).  ``A`` is formed in FP64 and
then rounded to the run dtype; the oracle is given that rounded matrix promoted back to FP64.

Storage convention (the library's): each matrix is column-major with leading dimension ``ld``.
A uniform batch is a C-order array of shape (batch, n, ld): entry (i, j) of matrix b is
``arr[b, j, i]``.  An uneven batch is one flat array plus per-matrix element offsets.

Randomness: numpy's Philox counter-based bit generator keyed by (base seed, workload id, stream
tag) and the matrix index, so any single matrix can be regenerated on its own.  Normal deviates
come from the raw 64-bit words by Box-Muller, which keeps the bytes independent of numpy's
version-dependent distribution code.
"""
from __future__ import annotations

import math
import os
from concurrent.futures import ThreadPoolExecutor
from dataclasses import dataclass, field

import numpy as np

BASE_SEED = 1707051410

# stream tags (second key word) -- one independent stream per purpose
TAG_U, TAG_V, TAG_SIGMA, TAG_SHAPE, TAG_MISC = 1, 2, 3, 4, 5


def _bitgen(workload: int, index: int, tag: int) -> np.random.Philox:
    key0 = (BASE_SEED << 16) | ((workload & 0xFF) << 8) | (tag & 0xFF)
    return np.random.Philox(key=[key0, int(index) & 0xFFFFFFFFFFFFFFFF])


def uniforms(workload: int, index: int, tag: int, count: int) -> np.ndarray:
    """``count`` uniforms in (0, 1) from 53-bit fractions of raw Philox words."""
    raw = _bitgen(workload, index, tag).random_raw(count)
    return ((raw >> np.uint64(11)).astype(np.float64) + 0.5) * 2.0 ** -53


def normals(workload: int, index: int, tag: int, count: int) -> np.ndarray:
    """``count`` standard normal deviates (Box-Muller on pairs of uniforms)."""
    half = (count + 1) // 2
    u = uniforms(workload, index, tag, 2 * half)
    r = np.sqrt(-2.0 * np.log(u[0::2]))
    th = 2.0 * np.pi * u[1::2]
    z = np.empty(2 * half)
    z[0::2] = r * np.cos(th)
    z[1::2] = r * np.sin(th)
    return z[:count]


def _haar_stack(gauss: np.ndarray) -> np.ndarray:
    """Orthonormal factors from a stack of Gaussian (rows x cols) matrices, sign-fixed."""
    q, r = np.linalg.qr(gauss)
    d = np.sign(np.diagonal(r, axis1=-2, axis2=-1)).copy()
    d[d == 0] = 1.0
    return q * d[..., None, :]


# ----------------------------------------------------------------------------------------------
# spectra of the five workloads
# ----------------------------------------------------------------------------------------------

def sigma_fp64_32(k: int = 32) -> np.ndarray:
    """sigma_i = 10^(-8 i / 31), i = 0..31 (condition number 1e8)."""
    i = np.arange(k, dtype=np.float64)
    return 10.0 ** (-8.0 * i / 31.0)


def sigma_exp8(k: int) -> np.ndarray:
    """sigma_i = exp(-i / 8)."""
    return np.exp(-np.arange(k, dtype=np.float64) / 8.0)


def sigma_loguniform(workload: int, index: int, k: int, lo: float = 1e-6, hi: float = 1.0) -> np.ndarray:
    """iid log-uniform on [lo, hi], sorted descending."""
    u = uniforms(workload, index, TAG_SIGMA, k)
    s = np.exp(math.log(lo) + u * (math.log(hi) - math.log(lo)))
    return np.sort(s)[::-1].copy()


def sigma_decay(r0: float, k: int) -> np.ndarray:
    """sigma_i = exp(-i / r0)."""
    return np.exp(-np.arange(k, dtype=np.float64) / r0)


# ----------------------------------------------------------------------------------------------
# batches
# ----------------------------------------------------------------------------------------------

@dataclass
class UniformBatch:
    """A batch of equally sized matrices, column-major, ``a`` of shape (batch, n, ld)."""
    m: int
    n: int
    ld: int
    a: np.ndarray                 # run dtype, (batch, n, ld)
    sigma: np.ndarray             # FP64 (batch, min(m, n)), the generator's spectrum (descending)

    @property
    def batch(self) -> int:
        return self.a.shape[0]

    def a64(self, b: int) -> np.ndarray:
        """Matrix b as an FP64 (m, n) array (the rounded run-dtype input, promoted)."""
        return self.a[b, :, : self.m].T.astype(np.float64)


def uniform_batch(workload: int, batch: int, m: int, n: int, dtype, sigma_of, ld: int | None = None,
                  first: int = 0, chunk: int = 256) -> UniformBatch:
    """Matrices ``first .. first+batch-1`` of a workload with spectrum ``sigma_of(index) -> (k,)``."""
    ld = m if ld is None else ld
    k = min(m, n)
    out = np.zeros((batch, n, ld), dtype=dtype)
    sig = np.empty((batch, k))

    def one_chunk(c0):
        c1 = min(batch, c0 + chunk)
        idx = range(first + c0, first + c1)
        gu = np.stack([normals(workload, i, TAG_U, m * k).reshape(m, k) for i in idx])
        gv = np.stack([normals(workload, i, TAG_V, n * k).reshape(n, k) for i in idx])
        u = _haar_stack(gu)
        v = _haar_stack(gv)
        s = np.stack([np.asarray(sigma_of(i), dtype=np.float64) for i in idx])
        a = np.matmul(v, np.swapaxes(u * s[:, None, :], 1, 2))   # (b, n, m) = A^T in C order
        out[c0:c1, :, :m] = a.astype(dtype)
        sig[c0:c1] = s

    starts = list(range(0, batch, chunk))
    if len(starts) > 1:
        with ThreadPoolExecutor(max_workers=min(len(starts), os.cpu_count() or 1)) as ex:
            list(ex.map(one_chunk, starts))
    elif starts:
        one_chunk(0)
    return UniformBatch(m=m, n=n, ld=ld, a=out, sigma=sig)


@dataclass
class RaggedBatch:
    """Matrices of differing sizes packed in one flat array (each column-major, ld = m)."""
    m: np.ndarray                 # int32 (batch,)
    n: np.ndarray                 # int32 (batch,)
    offset: np.ndarray            # int64 (batch,) element offsets into ``flat``
    flat: np.ndarray              # run dtype
    sigma: list = field(default_factory=list)   # FP64 spectra (may be empty for kernel blocks)
    extra: dict = field(default_factory=dict)

    @property
    def batch(self) -> int:
        return len(self.m)

    def a64(self, b: int) -> np.ndarray:
        mb, nb, o = int(self.m[b]), int(self.n[b]), int(self.offset[b])
        return self.flat[o:o + mb * nb].reshape(nb, mb).T.astype(np.float64)


def _pack(ms, ns, dtype):
    sizes = np.asarray(ms, dtype=np.int64) * np.asarray(ns, dtype=np.int64)
    # keep every matrix 16-byte aligned (multiple of 4 FP32 elements)
    padded = (sizes + 3) // 4 * 4
    off = np.zeros(len(sizes), dtype=np.int64)
    off[1:] = np.cumsum(padded)[:-1]
    flat = np.zeros(int(padded.sum()), dtype=dtype)
    return off, flat


# ----------------------------------------------------------------------------------------------
# the five workloads (sizes as stated; ``batch`` may be reduced for parity tests)
# ----------------------------------------------------------------------------------------------

def fp64_32_graded(batch: int = 1000, first: int = 0) -> UniformBatch:
    """1000 x (32 x 32) FP64, sigma_i = 10^(-8 i/31): the plain Jacobi SVD and QR batch."""
    s = sigma_fp64_32()
    return uniform_batch(0, batch, 32, 32, np.float64, lambda i: s, first=first)


def svd64_exp8(batch: int = 20000, first: int = 0) -> UniformBatch:
    """20000 x (64 x 64) FP32, sigma_i = exp(-i/8)."""
    s = sigma_exp8(64)
    return uniform_batch(1, batch, 64, 64, np.float32, lambda i: s, first=first)


def qr128x32_exp8(batch: int = 20000, first: int = 0) -> UniformBatch:
    """20000 x (128 x 32) FP32, sigma_i = exp(-i/8), i = 0..31 (QR batch)."""
    s = sigma_exp8(32)
    return uniform_batch(101, batch, 128, 32, np.float32, lambda i: s, first=first)


def block512_loguniform(batch: int = 500, first: int = 0, size: int = 512) -> UniformBatch:
    """500 x (512 x 512) FP32, sigma iid log-uniform on [1e-6, 1]."""
    return uniform_batch(2, batch, size, size, np.float32,
                         lambda i: sigma_loguniform(2, i, size), first=first, chunk=16)


def rsvd_uneven_blocks(batch: int = 16384, first: int = 0, sizes=(64, 128, 256), eps: float = 1e-5,
                       dtype=np.float32) -> RaggedBatch:
    """Uneven blocks: m, n iid uniform on ``sizes``; sigma_i = exp(-i/r0), r0 ~ U[2, 12]; rounded to
    ``dtype`` (FP32 for the workload; FP64 for the FP64 path's tests).

    ``extra['r0']`` holds r0 and ``extra['rank_hint']`` the rank at which sigma falls to
    ``eps`` relative, min(ceil(r0 ln(1/eps)), min(m, n)).
    """
    sizes = np.asarray(sizes)
    ms, ns, r0s = [], [], []
    for i in range(first, first + batch):
        u = uniforms(3, i, TAG_SHAPE, 3)
        ms.append(int(sizes[min(int(u[0] * len(sizes)), len(sizes) - 1)]))
        ns.append(int(sizes[min(int(u[1] * len(sizes)), len(sizes) - 1)]))
        r0s.append(2.0 + 10.0 * u[2])
    off, flat = _pack(ms, ns, dtype)
    sig = []
    for b, i in enumerate(range(first, first + batch)):
        m, n, r0 = ms[b], ns[b], r0s[b]
        k = min(m, n)
        u = _haar_stack(normals(3, i, TAG_U, m * k).reshape(m, k))
        v = _haar_stack(normals(3, i, TAG_V, n * k).reshape(n, k))
        s = sigma_decay(r0, k)
        a = (u * s) @ v.T
        flat[off[b]:off[b] + m * n] = a.T.reshape(-1).astype(dtype)
        sig.append(s)
    hint = np.array([min(math.ceil(r0 * math.log(1.0 / eps)), min(m, n))
                     for m, n, r0 in zip(ms, ns, r0s)], dtype=np.int32)
    return RaggedBatch(m=np.array(ms, np.int32), n=np.array(ns, np.int32), offset=off, flat=flat,
                       sigma=sig, extra={"r0": np.array(r0s), "rank_hint": hint})


# ----------------------------------------------------------------------------------------------
# kernel blocks: admissible blocks of an exponential covariance kernel over 3D points
# ----------------------------------------------------------------------------------------------

def _kd_tree(pts: np.ndarray, leaf: int):
    """Median split along the widest side of each box; returns (perm, nodes) with nodes as
    (start, end, lo, hi, children) in the permuted order."""
    perm = np.arange(len(pts))
    nodes = []

    def build(start, end):
        p = pts[perm[start:end]]
        lo, hi = p.min(axis=0), p.max(axis=0)
        idx = len(nodes)
        nodes.append([start, end, lo, hi, None])
        if end - start > leaf:
            d = int(np.argmax(hi - lo))
            order = np.argsort(p[:, d], kind="stable")
            perm[start:end] = perm[start:end][order]
            mid = (start + end) // 2
            c0 = build(start, mid)
            c1 = build(mid, end)
            nodes[idx][4] = (c0, c1)
        return idx

    build(0, len(pts))
    return perm, nodes


def _admissible(a, b, eta):
    da = float(np.linalg.norm(a[3] - a[2]))
    db = float(np.linalg.norm(b[3] - b[2]))
    gap = np.maximum(0.0, np.maximum(a[2] - b[3], b[2] - a[3]))
    return min(da, db) <= eta * float(np.linalg.norm(gap))


def kernel_blocks_3d(n_points: int = 32768, seed_index: int = 0, leaf: int = 64, eta: float = 1.1, ell: float = 0.1,
              lo: int = 64, hi: int = 256, max_blocks: int | None = None) -> RaggedBatch:
    """Admissible blocks K(t, s) = exp(-|x - y| / ell) of the dual traversal of a k-d tree over
    ``n_points`` uniform points in the unit cube, kept when lo <= |t|, |s| <= hi."""
    u = uniforms(4, seed_index, TAG_MISC, 3 * n_points).reshape(n_points, 3)
    perm, nodes = _kd_tree(u, leaf)
    pts = u[perm]
    pairs = []
    stack = [(0, 0)]
    while stack:
        t, s = stack.pop()
        a, b = nodes[t], nodes[s]
        if _admissible(a, b, eta):
            if lo <= a[1] - a[0] <= hi and lo <= b[1] - b[0] <= hi:
                pairs.append((t, s))
            continue
        if a[4] is None or b[4] is None:
            continue                       # a dense (inadmissible) leaf: not part of this workload
        for c in a[4]:
            for d in b[4]:
                stack.append((c, d))
    pairs.sort()
    if max_blocks is not None:
        pairs = pairs[:max_blocks]
    ms = [nodes[t][1] - nodes[t][0] for t, _ in pairs]
    ns = [nodes[s][1] - nodes[s][0] for _, s in pairs]
    off, flat = _pack(ms, ns, np.float32)

    def one(i):
        t, s = pairs[i]
        x = pts[nodes[t][0]:nodes[t][1]]
        y = pts[nodes[s][0]:nodes[s][1]]
        d = np.sqrt(((x[:, None, :] - y[None, :, :]) ** 2).sum(-1))
        blk = np.exp(-d / ell)
        flat[off[i]:off[i] + blk.size] = blk.T.reshape(-1).astype(np.float32)

    with ThreadPoolExecutor(max_workers=os.cpu_count() or 1) as ex:
        list(ex.map(one, range(len(pairs)), chunksize=256))
    return RaggedBatch(m=np.array(ms, np.int32), n=np.array(ns, np.int32), offset=off, flat=flat,
                       extra={"pairs": pairs, "n_points": n_points, "eta": eta})
