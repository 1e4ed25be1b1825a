"""FP64 CPU oracle (test infrastructure only).

Python access to ``oracle.c``: plain FP64 Householder QR (Algorithm 1), cyclic one-sided Jacobi
SVD (Algorithm 2), Philox4x32-10 / Box-Muller sampling matrices and the randomized SVD
(Algorithm 4) of Boukaram et al. (2017), plus the FP64 reference for the learned rank predictor.

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg may import this
package.  It shares no code with the CUDA library and never imports it.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None

NOT_CONVERGED = 1 << 20


def build(force: bool = False) -> str:
    """Compile ``oracle.c`` with gcc into ``oracle/_build/liboracle.so`` (portable flags)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm", "-lpthread"],
                       check=True)
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            d, i, ll, p = ctypes.c_double, ctypes.c_int, ctypes.c_longlong, ctypes.c_void_p
            u32, u64 = ctypes.c_uint32, ctypes.c_uint64
            L.orc_nrm2.restype = d
            L.orc_nrm2.argtypes = [i, p, i]
            L.orc_house.argtypes = [i, p, p]
            L.orc_qr.restype = i
            L.orc_qr.argtypes = [i, i, p, i, p, i, p, i]
            L.orc_rot.restype = i
            L.orc_rot.argtypes = [d, d, d, d, p, p]
            L.orc_jacobi_svd.restype = i
            L.orc_jacobi_svd.argtypes = [i, i, p, i, d, i, p, p, i, p, i, p]
            L.orc_philox4x32_10.argtypes = [p, p, p]
            L.orc_gauss.restype = d
            L.orc_gauss.argtypes = [u64, u32, u32, u32, u32]
            L.orc_omega.argtypes = [u64, u32, u32, i, i, i, p]
            L.orc_range_basis.restype = i
            L.orc_range_basis.argtypes = [i, i, p, i, p, i, i, p]
            L.orc_rsvd_finish.restype = i
            L.orc_rsvd_finish.argtypes = [i, i, p, i, p, i, p, p, p]
            L.orc_rsvd.restype = i
            L.orc_rsvd.argtypes = [i, i, p, i, u64, u32, i, i, p, p, p]
            L.orc_trunc_rank.restype = i
            L.orc_trunc_rank.argtypes = [i, p, d, d]
            L.orc_post_est2.restype = d
            L.orc_post_est2.argtypes = [i, i, p, i, p, p, p, i, u64, u32, i]
            L.orc_budget_rank.restype = i
            L.orc_budget_rank.argtypes = [i, p, d, d, d]
            L.orc_rsvd_adaptive.restype = i
            L.orc_rsvd_adaptive.argtypes = [i, i, p, i, u64, u32, i, d, i, i, i, i, p, p, p, p, p]
            L.orc_rsvd_rank.restype = i
            L.orc_rsvd_rank.argtypes = [i, i, p, i, u64, u32, i, i, i, i, p, p, p]
            L.orc_qr_batch.argtypes = [i, p, p, p, p, p, p, p, p, p, i]
            L.orc_svd_batch.argtypes = [i, p, p, p, p, d, i, p, p, p, p, p, p, p, p, i]
            _lib = L
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _f64(a) -> np.ndarray:
    """Column-major FP64 copy of a 2-D array."""
    return np.asfortranarray(np.asarray(a, dtype=np.float64))


def default_threads() -> int:
    return max(1, len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count() or 1)


# ----------------------------------------------------------------------------------------------
# single-matrix calls
# ----------------------------------------------------------------------------------------------

def nrm2(x) -> float:
    x = np.ascontiguousarray(x, dtype=np.float64)
    return lib().orc_nrm2(x.size, _p(x), 1)


def house(x) -> np.ndarray:
    x = np.ascontiguousarray(x, dtype=np.float64)
    v = np.empty_like(x)
    lib().orc_house(x.size, _p(x), _p(v))
    return v


def qr(a):
    """Reduced Householder QR (Algorithm 1) of an m x n matrix, m >= n: returns (Q, R)."""
    a = _f64(a)
    m, n = a.shape
    q = np.zeros((m, n), order="F")
    r = np.zeros((n, n), order="F")
    rc = lib().orc_qr(m, n, _p(a), max(m, 1), _p(q), max(m, 1), _p(r), max(n, 1))
    if rc:
        raise ValueError(f"orc_qr: bad shape {a.shape}")
    return q, r


def rot(alpha: float, beta: float, gamma: float, tol: float):
    """rot(G) of Algorithm 2: (rotated?, c, s)."""
    c = ctypes.c_double(1.0)
    s = ctypes.c_double(0.0)
    f = lib().orc_rot(alpha, beta, gamma, tol, ctypes.byref(c), ctypes.byref(s))
    return bool(f), c.value, s.value


def svd(a, tol: float = -1.0, max_sweeps: int = 30):
    """Reduced SVD by one-sided Jacobi (Algorithm 2): (U, S, V, info, rotations)."""
    a = _f64(a)
    m, n = a.shape
    k = min(m, n)
    u = np.zeros((m, k), order="F")
    v = np.zeros((n, k), order="F")
    s = np.zeros(k)
    rots = ctypes.c_longlong(0)
    info = lib().orc_jacobi_svd(m, n, _p(a), max(m, 1), tol, max_sweeps, _p(s), _p(u), max(m, 1),
                                _p(v), max(n, 1), ctypes.byref(rots))
    if info == -1:
        raise ValueError("orc_jacobi_svd: bad shape")
    return u, s, v, info, rots.value


def philox4x32_10(ctr, key) -> np.ndarray:
    c = np.asarray(ctr, dtype=np.uint32)
    k = np.asarray(key, dtype=np.uint32)
    o = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(_p(c), _p(k), _p(o))
    return o


def gauss(seed: int, index: int, tag: int, row: int, col: int) -> float:
    """Entry (row, col) of Gaussian stream `tag` of matrix `index` under `seed`."""
    return lib().orc_gauss(seed, index, tag, row, col)


def omega(seed: int, index: int, tag: int, n: int, c0: int, cols: int) -> np.ndarray:
    """Columns c0 .. c0+cols-1 of the Gaussian sampling stream (n rows)."""
    o = np.zeros((n, cols), order="F")
    lib().orc_omega(seed, index, tag, n, c0, cols, _p(o))
    return o


def range_basis(a, om, q: int) -> np.ndarray:
    a = _f64(a)
    om = _f64(om)
    m, n = a.shape
    l = om.shape[1]
    Q = np.zeros((m, l), order="F")
    rc = lib().orc_range_basis(m, n, _p(a), m, _p(om), l, q, _p(Q))
    if rc:
        raise ValueError("orc_range_basis failed")
    return Q


def rsvd_finish(a, Q):
    a = _f64(a)
    Q = _f64(Q)
    m, n = a.shape
    l = Q.shape[1]
    U = np.zeros((m, l), order="F")
    V = np.zeros((n, l), order="F")
    S = np.zeros(l)
    info = lib().orc_rsvd_finish(m, n, _p(a), m, _p(Q), l, _p(U), _p(S), _p(V))
    return U, S, V, info


def rsvd(a, seed: int, index: int, l: int, q: int = 1):
    """Fixed-width randomized SVD (Algorithm 4 with q power steps): (U, S, V, info)."""
    a = _f64(a)
    m, n = a.shape
    U = np.zeros((m, l), order="F")
    V = np.zeros((n, l), order="F")
    S = np.zeros(l)
    info = lib().orc_rsvd(m, n, _p(a), m, seed, index, l, q, _p(U), _p(S), _p(V))
    if info == -1:
        raise ValueError("orc_rsvd: need 1 <= l <= min(m, n)")
    return U, S, V, info


def trunc_rank(s, norm_a: float, eps: float) -> int:
    s = np.ascontiguousarray(s, dtype=np.float64)
    return lib().orc_trunc_rank(s.size, _p(s), norm_a, eps)


PROBES = 8


def post_est2(a, U, S, V, seed: int, index: int, r: int = PROBES) -> float:
    """Posterior estimate (Halko et al. 4.3) of ||A - U diag(S) V^T||_F^2 from r probes of stream 1."""
    a = _f64(a)
    m, n = a.shape
    U, V = _f64(U), _f64(V)
    S = np.ascontiguousarray(S, dtype=np.float64)
    l = S.size
    return lib().orc_post_est2(m, n, _p(a), m, _p(U), _p(S), _p(V), l, seed, index, r)


def budget_rank(s, norm2: float, eps: float, est2: float) -> int:
    """Smallest k with sum_{i>=k} s_i^2 <= (0.95 eps)^2 norm2 - 4 est2."""
    s = np.ascontiguousarray(s, dtype=np.float64)
    return lib().orc_budget_rank(s.size, _p(s), norm2, eps, est2)


def rsvd_adaptive(a, seed: int, index: int, hint: int = 0, eps: float = 1e-5, p: int = 8, q: int = 1,
                  max_rounds: int = 4, lcap: int = 128):
    """Adaptive randomized SVD to a relative Frobenius tolerance (rounds of p samples, posterior
    estimate, full-SVD fallback, budgeted truncation).  Returns a dict with U, S, V (first
    `samples` columns), rank, samples, rounds, fallback, est2, norm2 and est2_round."""
    a = _f64(a)
    m, n = a.shape
    k = min(m, n)
    U = np.zeros((m, k), order="F")
    V = np.zeros((n, k), order="F")
    S = np.zeros(k)
    res = np.zeros(6)
    er = np.full(max_rounds, np.nan)
    rc = lib().orc_rsvd_adaptive(m, n, _p(a), m, seed, index, int(hint), eps, p, q, max_rounds, lcap,
                                 _p(U), _p(S), _p(V), _p(res), _p(er))
    if rc:
        raise ValueError("orc_rsvd_adaptive: bad arguments")
    l = int(res[1])
    return {"U": U[:, :l], "S": S[:l], "V": V[:, :l], "rank": int(res[0]), "samples": l, "rounds": int(res[2]),
            "fallback": bool(res[3]), "est2": float(res[4]), "norm2": float(res[5]),
            "est2_round": er[:int(res[2])]}


def rsvd_rank(a, seed: int, index: int, k: int, p: int = 8, q: int = 1, lcap: int = 128):
    """Fixed-rank randomized SVD (Algorithm 4: k + p samples, q power steps, first k columns kept;
    the full SVD when k + p reaches min(m, n) or exceeds lcap): (U_k, S_k, V_k, samples)."""
    a = _f64(a)
    m, n = a.shape
    kk = min(m, n)
    U = np.zeros((m, kk), order="F")
    V = np.zeros((n, kk), order="F")
    S = np.zeros(kk)
    l = lib().orc_rsvd_rank(m, n, _p(a), m, seed, index, int(k), p, q, lcap, _p(U), _p(S), _p(V))
    if l < 0:
        raise ValueError("orc_rsvd_rank: bad arguments")
    k = min(int(k), kk)
    return U[:, :k].copy(), S[:k].copy(), V[:, :k].copy(), l


# ----------------------------------------------------------------------------------------------
# batch calls over lists of FP64 matrices (threads over independent matrices)
# ----------------------------------------------------------------------------------------------

def _flatten(mats):
    ms = np.array([a.shape[0] for a in mats], dtype=np.int32)
    ns = np.array([a.shape[1] for a in mats], dtype=np.int32)
    sizes = ms.astype(np.int64) * ns
    off = np.zeros(len(mats), dtype=np.int64)
    off[1:] = np.cumsum(sizes)[:-1]
    flat = np.zeros(int(sizes.sum()) + 1)
    for a, o in zip(mats, off):
        flat[o:o + a.size] = np.asarray(a, dtype=np.float64).T.reshape(-1)
    return ms, ns, off, flat


def svd_batch(mats, tol: float = -1.0, max_sweeps: int = 30, nthreads: int | None = None):
    """Jacobi SVD of each FP64 matrix: lists (U, S, V) plus arrays info, rotations."""
    nthreads = nthreads or default_threads()
    ms, ns, offA, flat = _flatten(mats)
    ks = np.minimum(ms, ns).astype(np.int64)
    offS = np.concatenate([[0], np.cumsum(ks)[:-1]]).astype(np.int64)
    offU = np.concatenate([[0], np.cumsum(ms * ks)[:-1]]).astype(np.int64)
    offV = np.concatenate([[0], np.cumsum(ns * ks)[:-1]]).astype(np.int64)
    S = np.zeros(int(ks.sum()) + 1)
    U = np.zeros(int((ms * ks).sum()) + 1)
    V = np.zeros(int((ns * ks).sum()) + 1)
    info = np.zeros(len(mats), dtype=np.int32)
    rots = np.zeros(len(mats), dtype=np.int64)
    lib().orc_svd_batch(len(mats), _p(ms), _p(ns), _p(flat), _p(offA), tol, max_sweeps, _p(S), _p(offS),
                        _p(U), _p(offU), _p(V), _p(offV), _p(info), _p(rots), nthreads)
    Us, Ss, Vs = [], [], []
    for b in range(len(mats)):
        m, n, k = int(ms[b]), int(ns[b]), int(ks[b])
        Ss.append(S[offS[b]:offS[b] + k].copy())
        Us.append(U[offU[b]:offU[b] + m * k].reshape(k, m).T.copy())
        Vs.append(V[offV[b]:offV[b] + n * k].reshape(k, n).T.copy())
    return Us, Ss, Vs, info, rots


def qr_batch(mats, nthreads: int | None = None):
    """Householder QR of each FP64 matrix (m >= n): lists (Q, R) plus info."""
    nthreads = nthreads or default_threads()
    ms, ns, offA, flat = _flatten(mats)
    offQ = offA.copy()
    n2 = ns.astype(np.int64) ** 2
    offR = np.concatenate([[0], np.cumsum(n2)[:-1]]).astype(np.int64)
    Q = np.zeros_like(flat)
    R = np.zeros(int(n2.sum()) + 1)
    info = np.zeros(len(mats), dtype=np.int32)
    lib().orc_qr_batch(len(mats), _p(ms), _p(ns), _p(flat), _p(offA), _p(Q), _p(offQ), _p(R), _p(offR),
                       _p(info), nthreads)
    Qs, Rs = [], []
    for b in range(len(mats)):
        m, n = int(ms[b]), int(ns[b])
        Qs.append(Q[offQ[b]:offQ[b] + m * n].reshape(n, m).T.copy())
        Rs.append(R[offR[b]:offR[b] + n * n].reshape(n, n).T.copy())
    return Qs, Rs, info
