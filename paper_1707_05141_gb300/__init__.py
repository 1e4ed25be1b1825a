"""GB300-native batched QR, one-sided Jacobi SVD and randomized SVD.

After Boukaram, Turkiyyah, Ltaief & Keyes, "Batched QR and SVD Algorithms on GPUs with
Applications in Hierarchical Matrix Compression" (2017).  The work happens in ``libbsvd.so``, a
CUDA library for sm_103a with the C ABI of ``include/bsvd.h``; this module only marshals
arguments to it through ctypes.  PyTorch supplies device memory and streams.  There is no CPU
path: every function raises if the library is not built or no CUDA device is present.
"""
from __future__ import annotations

import ctypes
import os
import threading

from .build import LIB, build  # noqa: F401  (build() compiles libbsvd.so in-tree)

F32, F64 = 0, 1
SUCCESS = 0
ERR_UNSUPPORTED = -1000
ERR_CUDA = -1001
ERR_WORKSPACE = -1002
ERR_SCRATCH_LIMIT = -1003
NOALLOC_SCRATCH_BYTES = 64 << 20
BLOCK_GRAM, BLOCK_DIRECT = 0, 1
INFO_BAD_SHAPE = -1
INFO_NOT_CONVERGED = 1 << 20
INFO_NO_SCRATCH = -2
INFO_RANK_CAPPED = 1 << 21
INFO_FALLBACK = 1 << 22
INFO_DEVICE_TIMEOUT = -3
INFO_NONFINITE = -4
RSVD_SMALL_FP64 = 1
RSVD_TC_SAMPLING = 2
BLOCK_SIMT_PRODUCTS = 1 << 16
BLOCK_TEST_TIMEOUT = 1 << 17
BLOCK_QR_PRECONDITION = 1 << 18
BLOCK_RETEST_ALL = 1 << 19
TIER_AUTO, TIER_REGISTER, TIER_SHARED = 0, 1, 2

_lock = threading.Lock()
_lib = None


class BsvdError(RuntimeError):
    """A non-zero status returned by an entry point of libbsvd.so."""

    def __init__(self, fn: str, code: int):
        what = {ERR_UNSUPPORTED: "unsupported shape", ERR_CUDA: "CUDA launch failure",
                ERR_WORKSPACE: "workspace too small", ERR_SCRATCH_LIMIT: "beyond the fixed scratch"}.get(code)
        super().__init__(f"{fn} returned {code}" + (f" ({what})" if what else f" (argument {-code} invalid)"))
        self.code = code


def lib() -> ctypes.CDLL:
    """The loaded CUDA library (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB):
                raise RuntimeError(f"{LIB} is missing: build it with paper_1707_05141_gb300.build()")
            L = ctypes.CDLL(LIB)
            i, d, p, ll = ctypes.c_int, ctypes.c_double, ctypes.c_void_p, ctypes.c_longlong
            L.bsvd_version.restype = ctypes.c_char_p
            L.bsvd_version.argtypes = []
            L.batched_qr.restype = i
            L.batched_qr.argtypes = [i, i, i, i, p, p, p, p, p, p, p, p, p, p]
            L.batched_qr_blocked_workspace.restype = ctypes.c_size_t
            L.batched_qr_blocked_workspace.argtypes = [i, i, i, i]
            L.batched_qr_blocked.restype = i
            L.batched_qr_blocked.argtypes = [i, i, i, i, p, p, p, p, p, p, p, p, p, p, ctypes.c_size_t, p]
            L.batched_qr_blocked_max_rows.restype = i
            L.batched_qr_blocked_max_rows.argtypes = [i]
            L.batched_svd_jacobi.restype = i
            L.batched_svd_jacobi.argtypes = [i, i, i, i, p, p, p, p, p, p, p, p, p, d, i, i, p, p, p]
            L.bsvd_set_block_choice.restype = i
            L.bsvd_set_block_choice.argtypes = [i, i, i, i, i]
            L.bsvd_jacobi_variants.restype = i
            L.bsvd_jacobi_variants.argtypes = [i, i, i, i]
            L.bsvd_jacobi_variant_desc.restype = i
            L.bsvd_jacobi_variant_desc.argtypes = [i, i, i, i, p]
            L.bsvd_set_jacobi_choice.restype = i
            L.bsvd_set_jacobi_choice.argtypes = [i, i, i, i]
            L.batched_svd_block_jacobi_workspace.restype = ctypes.c_size_t
            L.batched_svd_block_jacobi_workspace.argtypes = [i, i, i, i, i, i]
            L.batched_svd_block_jacobi.restype = i
            L.batched_svd_block_jacobi.argtypes = [i, i, i, i, p, p, p, p, p, p, p, p, p, d, i, i, i, p, p, p,
                                                   ctypes.c_size_t, p]
            L.batched_rsvd_workspace.restype = ctypes.c_size_t
            L.batched_rsvd_workspace.argtypes = [i, i, i, i, p, p]
            L.bsvd_h2_truncate_workspace.restype = ctypes.c_size_t
            L.bsvd_h2_truncate_workspace.argtypes = [i, i, i, i]
            L.bsvd_h2_truncate.restype = i
            L.bsvd_h2_truncate.argtypes = [i, i, i, i, p, p, p, p, d, p, p, p, p, p, p, p, p, ctypes.c_size_t, p]
            L.bsvd_host_svd_workspace.restype = ctypes.c_size_t
            L.bsvd_host_svd_workspace.argtypes = [i, i, i, i]
            L.bsvd_host_svd.restype = i
            L.bsvd_host_svd.argtypes = [i, i, i, i, p, p, p, p, p, i, p, ctypes.c_size_t, p]
            L.bsvd_host_qr_workspace.restype = ctypes.c_size_t
            L.bsvd_host_qr_workspace.argtypes = [i, i, i, i]
            L.bsvd_host_qr.restype = i
            L.bsvd_host_qr.argtypes = [i, i, i, i, p, p, p, p, i, p, ctypes.c_size_t, p]
            L.bsvd_philox_gauss.restype = i
            L.bsvd_philox_gauss.argtypes = [i, p, ctypes.c_ulonglong, p, p, p, p]
            L.bsvd_fma_probe.restype = ctypes.c_longlong
            L.bsvd_fma_probe.argtypes = [i, i, i, p, p]
            L.batched_rsvd.restype = i
            L.batched_rsvd.argtypes = [i, i, i, i, p, p, p, p, p, p, p, d, i, i, i, ctypes.c_ulonglong, i, p, p, p,
                                       p, p, p, p, p, p, p, p, ctypes.c_size_t, p]
            L.bsvd_sketch_features.restype = i
            L.bsvd_sketch_features.argtypes = [i, i, i, p, p, p, p, ctypes.c_ulonglong, p, p]
            L.bsvd_mlp_forward.restype = i
            L.bsvd_mlp_forward.argtypes = [i, p, p, p, p, ctypes.c_float, p, p, p]
            L.bsvd_mlp_grad.restype = i
            L.bsvd_mlp_grad.argtypes = [i, p, p, p, p, p, p]
            L.bsvd_mlp_adam.restype = i
            L.bsvd_mlp_adam.argtypes = [i, p, p, p, p, i, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                                        ctypes.c_float, p]
            L.bsvd_mlp_param_count.restype = i
            L.bsvd_mlp_param_count.argtypes = []
            L.batched_svd_block_jacobi_noalloc.restype = i
            L.batched_svd_block_jacobi_noalloc.argtypes = [i, i, i, i, p, p, p, p, p, p, p, p, p, d, i, i, i, p, p,
                                                           p]
            _lib = L
    return _lib


def version() -> str:
    return lib().bsvd_version().decode()


def jacobi_variants(dtype_code: int, max_m: int, max_n: int, tier: int) -> int:
    """Number of kernel variants of ``tier`` able to run a max_m x max_n batch."""
    return lib().bsvd_jacobi_variants(dtype_code, max_m, max_n, tier)


def jacobi_variant_desc(dtype_code: int, max_m: int, max_n: int, k: int) -> dict:
    """Shape parameters of the k-th (k >= 1) register-tier variant fitting max_m x max_n."""
    d = (ctypes.c_int * 9)()
    _check("bsvd_jacobi_variant_desc", lib().bsvd_jacobi_variant_desc(dtype_code, max_m, max_n, k, d))
    return dict(zip(("slots", "parts", "rows_a", "rows_v", "ctas_per_sm", "scaled", "qr_precond", "fp64_params",
                     "carried_norms"), list(d)))


def set_block_choice(dtype_code: int, max_m: int, max_n: int, block_width: int, inner_variant: int = 0) -> None:
    """Record the block width and inner variant that block_width = 0 uses for this size bin."""
    _check("bsvd_set_block_choice", lib().bsvd_set_block_choice(dtype_code, max_m, max_n, block_width, inner_variant))


def set_jacobi_choice(dtype_code: int, max_m: int, max_n: int, tier: int) -> None:
    """Record the (tier | variant << 8) that TIER_AUTO uses for this size bin."""
    _check("bsvd_set_jacobi_choice", lib().bsvd_set_jacobi_choice(dtype_code, max_m, max_n, tier))


# ----------------------------------------------------------------------------------------------
# marshalling helpers (torch is only the allocator)
# ----------------------------------------------------------------------------------------------

def _torch():
    import torch
    return torch


def _stream_ptr(stream):
    torch = _torch()
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(int(getattr(stream, "cuda_stream", stream)))


def _ptr(t):
    return ctypes.c_void_p(0 if t is None else int(t.data_ptr()))


def _dptr(t, name: str, dtype=None, numel: int = 0):
    """Device pointer of a caller's tensor (None: null), after the checks the kernels cannot make
    themselves: a host tensor, another element type or too few elements would have them read or
    write outside the tensor."""
    if t is None:
        return ctypes.c_void_p(0)
    torch = _torch()
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise ValueError(f"{name}: a CUDA tensor is required (the library takes device pointers)")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"{name}: {dtype} required, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name}: a contiguous tensor is required")
    if t.numel() < numel:
        raise ValueError(f"{name}: at least {numel} elements required, got {t.numel()}")
    return ctypes.c_void_p(int(t.data_ptr()))


def _same(X, A, name: str):
    """An output batch must hold A's element type and a pointer for every matrix of A."""
    if X is None:
        return
    if X.dtype != A.dtype:
        raise TypeError(f"{name}: {A.dtype} matrices required (the input's type), got {X.dtype}")
    if X.batch < A.batch:
        raise ValueError(f"{name}: {A.batch} matrices required, got {X.batch}")


class Batch:
    """A batch of column-major matrices in device memory, in the pointer-array form of the C ABI.

    ``ptrs`` (int64), ``m``, ``n``, ``ld`` (int32) are device tensors with one entry per matrix;
    ``max_m``/``max_n`` are host bounds.  ``keep`` holds the tensors that own the storage.
    """

    def __init__(self, ptrs, m, n, ld, dtype, max_m, max_n, keep=()):
        torch = _torch()
        if dtype not in (torch.float32, torch.float64):
            raise TypeError(f"matrices must be float32 or float64, got {dtype}")
        for t in (ptrs, m, n, ld):
            if not t.is_cuda:
                raise ValueError("a batch lives in device memory: CUDA tensors are required")
        self.ptrs, self.m, self.n, self.ld = ptrs, m, n, ld
        self.dtype, self.max_m, self.max_n = dtype, int(max_m), int(max_n)
        self.keep = tuple(keep)

    @property
    def batch(self) -> int:
        return int(self.ptrs.numel())

    @property
    def code(self) -> int:
        torch = _torch()
        return F32 if self.dtype == torch.float32 else F64

    @classmethod
    def uniform(cls, t, m: int | None = None, n: int | None = None):
        """``t`` of shape (batch, cols, ld), contiguous on the GPU: matrix b is t[b].T[:m, :n]."""
        torch = _torch()
        if not (t.is_cuda and t.is_contiguous() and t.dim() == 3):
            raise ValueError("Batch.uniform: a contiguous 3-D CUDA tensor (batch, cols, ld) is required")
        bsz, cols, ld = t.shape
        m = ld if m is None else m
        n = cols if n is None else n
        es = t.element_size()
        base = int(t.data_ptr())
        dev = t.device
        ptrs = base + torch.arange(bsz, device=dev, dtype=torch.int64) * (cols * ld * es)
        full = lambda v: torch.full((bsz,), int(v), device=dev, dtype=torch.int32)
        return cls(ptrs, full(m), full(n), full(ld), t.dtype, m, n, keep=(t,))

    @classmethod
    def packed(cls, flat, offsets, m, n, ld=None):
        """Matrices at element ``offsets`` of a flat device tensor; ``m``, ``n``, ``ld`` per matrix
        (``ld`` defaults to max(1, m))."""
        torch = _torch()
        if not flat.is_cuda:
            raise ValueError("Batch.packed: the flat storage must be a CUDA tensor")
        dev = flat.device
        off = torch.as_tensor(offsets, dtype=torch.int64).to(dev)
        mt = torch.as_tensor(m, dtype=torch.int32).to(dev)
        nt = torch.as_tensor(n, dtype=torch.int32).to(dev)
        ldt = mt.clamp(min=1) if ld is None else torch.as_tensor(ld, dtype=torch.int32).to(dev)
        ptrs = int(flat.data_ptr()) + off * flat.element_size()
        mh = torch.as_tensor(m)
        nh = torch.as_tensor(n)
        return cls(ptrs, mt, nt, ldt, flat.dtype, int(mh.max()) if mh.numel() else 0,
                   int(nh.max()) if nh.numel() else 0, keep=(flat,))


def _check(fn, rc):
    if rc != SUCCESS:
        raise BsvdError(fn, rc)


# ----------------------------------------------------------------------------------------------
# entry points (same names as the C ABI)
# ----------------------------------------------------------------------------------------------

def batched_qr(A: Batch, Q: Batch | None, R: Batch | None, info, stream=None) -> None:
    """Reduced Householder QR of every matrix of ``A`` (Algorithm 1); see include/bsvd.h."""
    torch = _torch()
    _same(Q, A, "Q")
    _same(R, A, "R")
    rc = lib().batched_qr(A.code, A.batch, A.max_m, A.max_n, _ptr(A.ptrs), _ptr(A.m), _ptr(A.n), _ptr(A.ld),
                          _ptr(Q.ptrs if Q else None), _ptr(Q.ld if Q else None),
                          _ptr(R.ptrs if R else None), _ptr(R.ld if R else None),
                          _dptr(info, "info", torch.int32, A.batch), _stream_ptr(stream))
    _check("batched_qr", rc)


def batched_qr_blocked_workspace(A: Batch) -> int:
    """Workspace bytes batched_qr_blocked needs for this batch's bounds."""
    return int(lib().batched_qr_blocked_workspace(A.code, A.batch, A.max_m, A.max_n))


def batched_qr_blocked_max_rows(dtype_code: int) -> int:
    """The tallest matrix batched_qr_blocked factors."""
    return int(lib().batched_qr_blocked_max_rows(dtype_code))


def batched_qr_blocked(A: Batch, Q: Batch | None, R: Batch | None, info, workspace, stream=None) -> None:
    """Blocked Householder QR (32-column panels, compact WY updates) of matrices beyond batched_qr's
    shared-memory kernel; ``workspace`` a device uint8 tensor.  See include/bsvd.h."""
    torch = _torch()
    _same(Q, A, "Q")
    _same(R, A, "R")
    nbytes = batched_qr_blocked_workspace(A)
    ws = _dptr(workspace, "workspace", torch.uint8, nbytes)
    rc = lib().batched_qr_blocked(A.code, A.batch, A.max_m, A.max_n, _ptr(A.ptrs), _ptr(A.m), _ptr(A.n),
                                  _ptr(A.ld), _ptr(Q.ptrs if Q else None), _ptr(Q.ld if Q else None),
                                  _ptr(R.ptrs if R else None), _ptr(R.ld if R else None),
                                  _dptr(info, "info", torch.int32, A.batch), ws, workspace.numel(),
                                  _stream_ptr(stream))
    _check("batched_qr_blocked", rc)


def batched_svd_jacobi(A: Batch, S: Batch, U: Batch | None, V: Batch | None, info, rotations=None,
                       tol: float = 0.0, max_sweeps: int = 0, tier: int = TIER_AUTO, stream=None) -> None:
    """Reduced SVD of every matrix of ``A`` by one-sided Jacobi (Algorithm 2); see include/bsvd.h."""
    torch = _torch()
    for X, name in ((S, "S"), (U, "U"), (V, "V")):
        _same(X, A, name)
    rc = lib().batched_svd_jacobi(A.code, A.batch, A.max_m, A.max_n, _ptr(A.ptrs), _ptr(A.m), _ptr(A.n), _ptr(A.ld),
                                  _ptr(S.ptrs), _ptr(U.ptrs if U else None), _ptr(U.ld if U else None),
                                  _ptr(V.ptrs if V else None), _ptr(V.ld if V else None), float(tol),
                                  int(max_sweeps), int(tier), _dptr(info, "info", torch.int32, A.batch),
                                  _dptr(rotations, "rotations", torch.int64, A.batch), _stream_ptr(stream))
    _check("batched_svd_jacobi", rc)


def batched_svd_block_jacobi_workspace(A: Batch, block_width: int = 32, method: int = BLOCK_GRAM) -> int:
    """Workspace bytes batched_svd_block_jacobi needs for this batch's bounds."""
    return int(lib().batched_svd_block_jacobi_workspace(A.code, A.batch, A.max_m, A.max_n, block_width, method))


def batched_svd_block_jacobi(A: Batch, S: Batch, U: Batch, V: Batch, info, workspace, rotations=None,
                             tol: float = 0.0, max_sweeps: int = 0, block_width: int = 32,
                             method: int = BLOCK_GRAM, stream=None) -> None:
    """Reduced SVD by one-sided block Jacobi (Algorithm 3); ``workspace`` a device uint8 tensor."""
    torch = _torch()
    for X, name in ((S, "S"), (U, "U"), (V, "V")):
        _same(X, A, name)
    rc = lib().batched_svd_block_jacobi(A.code, A.batch, A.max_m, A.max_n, _ptr(A.ptrs), _ptr(A.m), _ptr(A.n),
                                        _ptr(A.ld), _ptr(S.ptrs), _ptr(U.ptrs), _ptr(U.ld), _ptr(V.ptrs), _ptr(V.ld),
                                        float(tol), int(max_sweeps), int(block_width), int(method),
                                        _dptr(info, "info", torch.int32, A.batch),
                                        _dptr(rotations, "rotations", torch.int64, A.batch),
                                        _dptr(workspace, "workspace", torch.uint8), int(workspace.numel()),
                                        _stream_ptr(stream))
    _check("batched_svd_block_jacobi", rc)


def batched_rsvd_workspace(A: Batch, h_m=None, h_n=None) -> int:
    """Workspace bytes batched_rsvd needs (host size arrays give the exact size)."""
    import numpy as np
    hm = None if h_m is None else np.ascontiguousarray(h_m, dtype=np.int32)
    hn = None if h_n is None else np.ascontiguousarray(h_n, dtype=np.int32)
    return int(lib().batched_rsvd_workspace(A.code, A.batch, A.max_m, A.max_n,
                                            None if hm is None else hm.ctypes.data_as(ctypes.c_void_p),
                                            None if hn is None else hn.ctypes.data_as(ctypes.c_void_p)))


def batched_rsvd(A: Batch, U: Batch, S: Batch, V: Batch, kmax, rank, info, workspace, rank_hint=None,
                 tol: float = 1e-5, oversample: int = 8, max_rounds: int = 4, seed: int = 0, err_est=None,
                 samples=None, stream=None, fixed_rank=None, tol_per=None, power_iters: int = 1,
                 flags: int = 0) -> None:
    """Randomized SVD (Algorithm 4 + q power steps), fixed-rank (``fixed_rank`` > 0) or to a
    tolerance (``tol``, or ``tol_per`` per matrix); see include/bsvd.h."""
    torch = _torch()
    for X, name in ((S, "S"), (U, "U"), (V, "V")):
        _same(X, A, name)
    nb, i32 = A.batch, torch.int32
    rc = lib().batched_rsvd(A.code, A.batch, A.max_m, A.max_n, _ptr(A.ptrs), _ptr(A.m), _ptr(A.n), _ptr(A.ld),
                            _dptr(fixed_rank, "fixed_rank", i32, nb), _dptr(rank_hint, "rank_hint", i32, nb),
                            _dptr(tol_per, "tol_per", torch.float64, nb), float(tol), int(oversample),
                            int(power_iters), int(max_rounds), int(seed), int(flags), _ptr(U.ptrs), _ptr(U.ld),
                            _ptr(S.ptrs),
                            _ptr(V.ptrs), _ptr(V.ld), _dptr(kmax, "kmax", i32, nb), _dptr(rank, "rank", i32, nb),
                            _dptr(err_est, "err_est", torch.float32, nb), _dptr(samples, "samples", i32, nb),
                            _dptr(info, "info", i32, nb), _dptr(workspace, "workspace", torch.uint8),
                            int(workspace.numel()), _stream_ptr(stream))
    _check("batched_rsvd", rc)


class H2Plan:
    """A basis tree staged on the GPU for ``bsvd_h2_truncate`` (Section 8.2): leaves packed in one
    flat device tensor (column-major at ``offsets``), transfers and the outputs as (nodes, k, k)
    tensors (node g's matrix column-major: tensor[g].T), heap order (node i of level l is
    2^l - 1 + i), the workspace allocated once.  ``run`` truncates to ``eps``."""

    def __init__(self, leaves, transfers, k: int, dtype=None):
        import numpy as np
        torch = _torch()
        dt = torch.float32 if dtype in (None, np.float32, torch.float32) else torch.float64
        npdt = np.float32 if dt == torch.float32 else np.float64
        dev = torch.device("cuda")
        d = len(transfers) - 1
        nl = len(leaves)
        if nl != 2 ** d:
            raise ValueError("a tree of depth d has 2^d leaves")
        nodes = 2 * nl - 1
        ms = np.array([np.asarray(u).shape[0] for u in leaves], dtype=np.int32)
        lds = np.maximum(ms, 1).astype(np.int32)
        sizes = (lds.astype(np.int64) * k + 3) // 4 * 4
        offs = np.concatenate([[0], np.cumsum(sizes)[:-1]]).astype(np.int64)
        flat = np.zeros(int(sizes.sum()) + 4, dtype=npdt)
        for u, o, m in zip(leaves, offs, ms):
            flat[o:o + m * k] = np.asarray(u, dtype=np.float64).T.reshape(-1).astype(npdt)
        E = np.zeros((nodes, k, k), dtype=npdt)
        for l in range(1, d + 1):
            for i, e in enumerate(transfers[l]):
                E[2 ** l - 1 + i] = np.asarray(e, dtype=np.float64).T.astype(npdt)   # column-major
        self.leaf = torch.from_numpy(flat).to(dev)
        self.new_leaf = torch.zeros_like(self.leaf)
        self.E = torch.from_numpy(E).to(dev)
        self.new_transfer = torch.zeros_like(self.E)
        self.T = torch.zeros_like(self.E)
        self.rank = torch.zeros(nodes, dtype=torch.int32, device=dev)
        self.info = torch.zeros(nodes, dtype=torch.int32, device=dev)
        self.rotations = torch.zeros(nodes, dtype=torch.int64, device=dev)
        es = self.leaf.element_size()
        self.leaf_p = torch.as_tensor(offs * es + int(self.leaf.data_ptr()), dtype=torch.int64).to(dev)
        self.new_leaf_p = torch.as_tensor(offs * es + int(self.new_leaf.data_ptr()), dtype=torch.int64).to(dev)
        node_off = torch.arange(nodes, dtype=torch.int64, device=dev) * (k * k * es)
        self.E_p = node_off + int(self.E.data_ptr())
        self.newE_p = node_off + int(self.new_transfer.data_ptr())
        self.T_p = node_off + int(self.T.data_ptr())
        self.m_d = torch.as_tensor(ms).to(dev)
        self.ld_d = torch.as_tensor(lds).to(dev)
        self.code = F32 if dt == torch.float32 else F64
        self.max_m = int(ms.max()) if nl else 0
        self.depth, self.k, self.m, self.offsets, self.nodes = d, k, ms, offs, nodes
        self.workspace = torch.empty(int(lib().bsvd_h2_truncate_workspace(self.code, d, k, self.max_m)),
                                     dtype=torch.uint8, device=dev)

    def run(self, eps: float, stream=None) -> None:
        torch = _torch()
        rc = lib().bsvd_h2_truncate(self.code, self.depth, self.k, self.max_m, _ptr(self.leaf_p), _ptr(self.m_d),
                                    _ptr(self.ld_d), _ptr(self.E_p), float(eps), _ptr(self.new_leaf_p),
                                    _ptr(self.ld_d), _ptr(self.newE_p), _ptr(self.T_p), _ptr(self.rank),
                                    _ptr(self.info), _ptr(self.rotations),
                                    _dptr(self.workspace, "workspace", torch.uint8), int(self.workspace.numel()),
                                    _stream_ptr(stream))
        _check("bsvd_h2_truncate", rc)


def h2_truncate(leaves, transfers, k: int, eps: float, dtype=None, stream=None):
    """Truncation phase of H^2 compression (Section 8.2) on the GPU; returns the H2Plan holding the
    outputs (``new_leaf``, ``new_transfer``, ``T``, ``rank``, ``info``, ``rotations``)."""
    plan = H2Plan(leaves, transfers, k, dtype)
    plan.run(eps, stream)
    return plan


def _host_ptr(t, name: str, dtype, numel: int):
    """Address of a host tensor's data (None: null) after checks of device, type and size."""
    if t is None:
        return ctypes.c_void_p(0)
    torch = _torch()
    if not isinstance(t, torch.Tensor) or t.is_cuda:
        raise ValueError(f"{name}: a host tensor is required")
    if t.dtype != dtype:
        raise TypeError(f"{name}: {dtype} required, got {t.dtype}")
    if not t.is_contiguous() or t.numel() < numel:
        raise ValueError(f"{name}: a contiguous tensor of at least {numel} elements is required")
    return ctypes.c_void_p(int(t.data_ptr()))


def host_svd_workspace(dtype_code: int, batch: int, m: int, n: int) -> int:
    return int(lib().bsvd_host_svd_workspace(dtype_code, batch, m, n))


def host_svd(a, s, u=None, v=None, info=None, chunks: int = 4, workspace=None, stream=None) -> None:
    """Jacobi SVD of the host batch ``a`` (batch, n, m) into host ``s`` (batch, k), ``u`` (batch, k, m),
    ``v`` (batch, k, n), ``info`` (batch) int32, copies overlapped with the computation in ``chunks``
    chunks; ``workspace`` a uint8 CUDA tensor of host_svd_workspace(...) bytes."""
    torch = _torch()
    bsz, n, m = a.shape
    k = min(m, n)
    code = F32 if a.dtype == torch.float32 else F64
    rc = lib().bsvd_host_svd(code, bsz, m, n, _host_ptr(a, "a", a.dtype, bsz * m * n),
                             _host_ptr(s, "s", a.dtype, bsz * k), _host_ptr(u, "u", a.dtype, bsz * m * k),
                             _host_ptr(v, "v", a.dtype, bsz * n * k), _host_ptr(info, "info", torch.int32, bsz),
                             int(chunks), _dptr(workspace, "workspace", torch.uint8), int(workspace.numel()),
                             _stream_ptr(stream))
    _check("bsvd_host_svd", rc)


def host_qr_workspace(dtype_code: int, batch: int, m: int, n: int) -> int:
    return int(lib().bsvd_host_qr_workspace(dtype_code, batch, m, n))


def host_qr(a, q=None, r=None, info=None, chunks: int = 4, workspace=None, stream=None) -> None:
    """Householder QR of the host batch ``a`` (batch, n, m) into host ``q`` (batch, n, m), ``r``
    (batch, n, n), ``info`` (batch) int32, copies overlapped with the computation."""
    torch = _torch()
    bsz, n, m = a.shape
    code = F32 if a.dtype == torch.float32 else F64
    rc = lib().bsvd_host_qr(code, bsz, m, n, _host_ptr(a, "a", a.dtype, bsz * m * n),
                            _host_ptr(q, "q", a.dtype, bsz * m * n), _host_ptr(r, "r", a.dtype, bsz * n * n),
                            _host_ptr(info, "info", torch.int32, bsz), int(chunks),
                            _dptr(workspace, "workspace", torch.uint8), int(workspace.numel()), _stream_ptr(stream))
    _check("bsvd_host_qr", rc)


def philox_gauss(ctr, seed: int, stream=None):
    """Generator access for tests: (words uint32 [count, 4], FP32 Gaussians [count, 4], FP64 Gaussians
    [count, 4]) of the counters ``ctr`` (int64-compatible [count, 4]) under ``seed``."""
    import numpy as np
    torch = _torch()
    c = np.ascontiguousarray(np.asarray(ctr, dtype=np.uint64).reshape(-1, 4).astype(np.uint32).view(np.int32))
    cnt = c.shape[0]
    dev = torch.device("cuda")
    cu = torch.from_numpy(c).to(dev).contiguous()
    words = torch.zeros((cnt, 4), dtype=torch.int32, device=dev)
    g = torch.zeros((cnt, 4), dtype=torch.float32, device=dev)
    g64 = torch.zeros((cnt, 4), dtype=torch.float64, device=dev)
    rc = lib().bsvd_philox_gauss(cnt, _ptr(cu), int(seed), _ptr(words), _ptr(g), _ptr(g64), _stream_ptr(stream))
    _check("bsvd_philox_gauss", rc)
    return words, g, g64


def fma_probe(dtype_code: int, blocks: int, iters: int, out, stream=None) -> int:
    """Launch the FMA throughput probe; returns the flops it performs."""
    f = int(lib().bsvd_fma_probe(int(dtype_code), int(blocks), int(iters), _ptr(out), _stream_ptr(stream)))
    if f < 0:
        raise BsvdError("bsvd_fma_probe", f)
    return f


SKETCH_FEATURES = 16
MLP_PARAMS = 5313


def bsvd_sketch_features(A: Batch, features, seed: int = 0, stream=None) -> None:
    """16 sketch features per matrix into ``features`` (batch x 16 FP32 device tensor)."""
    torch = _torch()
    if A.dtype != torch.float32:
        raise TypeError("bsvd_sketch_features: float32 matrices required")
    feat = _dptr(features, "features", torch.float32, A.batch * SKETCH_FEATURES)
    _check("bsvd_sketch_features", lib().bsvd_sketch_features(A.batch, A.max_m, A.max_n, _ptr(A.ptrs), _ptr(A.m),
                                                               _ptr(A.n), _ptr(A.ld), int(seed), feat,
                                                               _stream_ptr(stream)))


def bsvd_mlp_forward(features, params, out=None, hint=None, margin: float = 2.0, m=None, n=None, stream=None):
    torch = _torch()
    batch = int(features.shape[0])
    f32, i32 = torch.float32, torch.int32
    _check("bsvd_mlp_forward", lib().bsvd_mlp_forward(batch, _dptr(features, "features", f32, batch * SKETCH_FEATURES),
                                                       _dptr(params, "params", f32, MLP_PARAMS),
                                                       _dptr(out, "out", f32, batch), _dptr(hint, "hint", i32, batch),
                                                       float(margin), _dptr(m, "m", i32, batch),
                                                       _dptr(n, "n", i32, batch), _stream_ptr(stream)))


def bsvd_mlp_grad(features, target, params, grad, loss, stream=None):
    torch = _torch()
    batch = int(features.shape[0])
    f32 = torch.float32
    _check("bsvd_mlp_grad", lib().bsvd_mlp_grad(batch, _dptr(features, "features", f32, batch * SKETCH_FEATURES),
                                                 _dptr(target, "target", f32, batch),
                                                 _dptr(params, "params", f32, MLP_PARAMS),
                                                 _dptr(grad, "grad", f32, MLP_PARAMS), _dptr(loss, "loss", f32, 1),
                                                 _stream_ptr(stream)))


def bsvd_mlp_adam(params, grad, mom, vel, step: int, lr: float = 1e-3, beta1: float = 0.9, beta2: float = 0.999,
                  eps: float = 1e-8, stream=None):
    torch = _torch()
    f32, npar = torch.float32, int(params.numel())
    _check("bsvd_mlp_adam", lib().bsvd_mlp_adam(npar, _dptr(params, "params", f32), _dptr(grad, "grad", f32, npar),
                                                 _dptr(mom, "mom", f32, npar), _dptr(vel, "vel", f32, npar),
                                                 int(step), float(lr), float(beta1), float(beta2), float(eps),
                                                 _stream_ptr(stream)))


class RsvdResult:
    """Outputs of ``rsvd``: flat device buffers plus per-matrix views on the host side."""

    def __init__(self, **kw):
        self.__dict__.update(kw)


def rsvd(flat, offsets, m, n, rank_hint=None, kmax=None, tol: float = 1e-5, oversample: int = 8,
         max_rounds: int = 4, seed: int = 0, stream=None, workspace=None, fixed_rank=None, tol_per=None,
         power_iters: int = 1, flags: int = 0):
    """Randomized SVD of matrices packed in ``flat`` (a device FP32 or FP64 tensor) at element
    ``offsets`` with sizes ``m``, ``n`` (host sequences).  Allocates the outputs (kmax columns each,
    default min(m, n)) and, unless given, the workspace."""
    import numpy as np
    torch = _torch()
    dev = flat.device
    m = np.asarray(m, dtype=np.int32)
    n = np.asarray(n, dtype=np.int32)
    bsz = len(m)
    k = np.minimum(m, n)
    km = k.copy() if kmax is None else np.asarray(kmax, dtype=np.int32)
    su = (m.astype(np.int64) * km + 3) // 4 * 4
    sv = (n.astype(np.int64) * km + 3) // 4 * 4
    ss = (km.astype(np.int64) + 3) // 4 * 4
    ou = np.concatenate([[0], np.cumsum(su)[:-1]])
    ov = np.concatenate([[0], np.cumsum(sv)[:-1]])
    os_ = np.concatenate([[0], np.cumsum(ss)[:-1]])
    fu = torch.zeros(int(su.sum()) + 4, device=dev, dtype=flat.dtype)
    fv = torch.zeros(int(sv.sum()) + 4, device=dev, dtype=flat.dtype)
    fs = torch.zeros(int(ss.sum()) + 4, device=dev, dtype=flat.dtype)
    A = Batch.packed(flat, offsets, m, n)
    U = Batch.packed(fu, ou, m, km)
    V = Batch.packed(fv, ov, n, km)
    S = Batch.packed(fs, os_, km, np.ones_like(km))
    kmax_d = torch.as_tensor(km, dtype=torch.int32).to(dev)

    def dev_array(x, dtype):
        if x is None:
            return None
        if isinstance(x, torch.Tensor):
            return x.to(device=dev, dtype=dtype).contiguous()
        return torch.as_tensor(np.asarray(x)).to(device=dev, dtype=dtype)

    hint_d = dev_array(rank_hint, torch.int32)
    fixed_d = dev_array(fixed_rank, torch.int32)
    tol_d = dev_array(tol_per, torch.float64)
    rank = torch.zeros(bsz, dtype=torch.int32, device=dev)
    info = torch.zeros(bsz, dtype=torch.int32, device=dev)
    err = torch.zeros(bsz, dtype=torch.float32, device=dev)
    samples = torch.zeros(bsz, dtype=torch.int32, device=dev)
    if workspace is None:
        workspace = torch.empty(batched_rsvd_workspace(A, m, n), dtype=torch.uint8, device=dev)
    batched_rsvd(A, U, S, V, kmax_d, rank, info, workspace, hint_d, tol, oversample, max_rounds, seed, err,
                 samples, stream, fixed_rank=fixed_d, tol_per=tol_d, power_iters=power_iters, flags=flags)
    return RsvdResult(U=fu, V=fv, S=fs, off_u=ou, off_v=ov, off_s=os_, kmax=km, rank=rank, info=info, err_est=err,
                      samples=samples, workspace=workspace, m=m, n=n)


def batched_svd_block_jacobi_noalloc(A: Batch, S: Batch, U: Batch, V: Batch, info, rotations=None,
                                     tol: float = 0.0, max_sweeps: int = 0, block_width: int = 32,
                                     method: int = BLOCK_GRAM, stream=None) -> None:
    """Block-Jacobi SVD with the library's own fixed scratch (no workspace, no allocation);
    see include/bsvd.h for its limit and the rule against overlapping calls."""
    torch = _torch()
    for X, name in ((S, "S"), (U, "U"), (V, "V")):
        _same(X, A, name)
    rc = lib().batched_svd_block_jacobi_noalloc(A.code, A.batch, A.max_m, A.max_n, _ptr(A.ptrs), _ptr(A.m),
                                                _ptr(A.n), _ptr(A.ld), _ptr(S.ptrs), _ptr(U.ptrs), _ptr(U.ld),
                                                _ptr(V.ptrs), _ptr(V.ld), float(tol), int(max_sweeps),
                                                int(block_width), int(method),
                                                _dptr(info, "info", torch.int32, A.batch),
                                                _dptr(rotations, "rotations", torch.int64, A.batch),
                                                _stream_ptr(stream))
    _check("batched_svd_block_jacobi_noalloc", rc)


# ----------------------------------------------------------------------------------------------
# conveniences that allocate the outputs with torch (uniform batches)
# ----------------------------------------------------------------------------------------------

def qr_blocked(a, want_q: bool = True, want_r: bool = True, stream=None):
    """Blocked QR of a uniform batch ``a`` (batch, n, m) -> (Q (batch, n, m), R (batch, n, n), info)."""
    torch = _torch()
    bsz, n, m = a.shape
    A = Batch.uniform(a.contiguous(), m, n)
    q = torch.empty((bsz, n, m), device=a.device, dtype=a.dtype) if want_q else None
    r = torch.empty((bsz, n, n), device=a.device, dtype=a.dtype) if want_r else None
    info = torch.empty(bsz, device=a.device, dtype=torch.int32)
    ws = torch.empty(max(batched_qr_blocked_workspace(A), 1), device=a.device, dtype=torch.uint8)
    batched_qr_blocked(A, Batch.uniform(q, m, n) if want_q else None, Batch.uniform(r, n, n) if want_r else None,
                       info, ws, stream)
    return q, r, info


def qr(a, want_q: bool = True, want_r: bool = True, stream=None):
    """QR of a uniform batch ``a`` (batch, n, m) on the GPU -> (Q (batch, n, m), R (batch, n, n), info)."""
    torch = _torch()
    bsz, n, m = a.shape
    A = Batch.uniform(a.contiguous(), m, n)
    q = torch.empty((bsz, n, m), device=a.device, dtype=a.dtype) if want_q else None
    r = torch.empty((bsz, n, n), device=a.device, dtype=a.dtype) if want_r else None
    info = torch.empty(bsz, device=a.device, dtype=torch.int32)
    batched_qr(A, Batch.uniform(q, m, n) if want_q else None, Batch.uniform(r, n, n) if want_r else None, info,
               stream)
    return q, r, info


def svd(a, want_u: bool = True, want_v: bool = True, tol: float = 0.0, max_sweeps: int = 0, tier: int = TIER_AUTO,
        stream=None):
    """Jacobi SVD of a uniform batch ``a`` (batch, n, m) -> (U (batch, k, m), S (batch, k), V (batch, k, n),
    info, rotations)."""
    torch = _torch()
    bsz, n, m = a.shape
    k = min(m, n)
    A = Batch.uniform(a.contiguous(), m, n)
    s = torch.empty((bsz, 1, k), device=a.device, dtype=a.dtype)
    u = torch.empty((bsz, k, m), device=a.device, dtype=a.dtype) if want_u else None
    v = torch.empty((bsz, k, n), device=a.device, dtype=a.dtype) if want_v else None
    info = torch.empty(bsz, device=a.device, dtype=torch.int32)
    rots = torch.empty(bsz, device=a.device, dtype=torch.int64)
    batched_svd_jacobi(A, Batch.uniform(s, k, 1), Batch.uniform(u, m, k) if want_u else None,
                       Batch.uniform(v, n, k) if want_v else None, info, rots, tol, max_sweeps, tier, stream)
    return u, s.view(bsz, k), v, info, rots


def svd_block(a, block_width: int = 32, method: int = BLOCK_GRAM, tol: float = 0.0, max_sweeps: int = 0,
              stream=None):
    """Block-Jacobi SVD of a uniform batch ``a`` (batch, n, m) -> (U, S, V, info, rotations)."""
    torch = _torch()
    bsz, n, m = a.shape
    k = min(m, n)
    A = Batch.uniform(a.contiguous(), m, n)
    s = torch.empty((bsz, 1, k), device=a.device, dtype=a.dtype)
    u = torch.empty((bsz, k, m), device=a.device, dtype=a.dtype)
    v = torch.empty((bsz, k, n), device=a.device, dtype=a.dtype)
    info = torch.empty(bsz, device=a.device, dtype=torch.int32)
    rots = torch.empty(bsz, device=a.device, dtype=torch.int64)
    ws = torch.empty(batched_svd_block_jacobi_workspace(A, block_width, method), device=a.device, dtype=torch.uint8)
    batched_svd_block_jacobi(A, Batch.uniform(s, k, 1), Batch.uniform(u, m, k), Batch.uniform(v, n, k), info, ws,
                             rots, tol, max_sweeps, block_width, method, stream)
    return u, s.view(bsz, k), v, info, rots
