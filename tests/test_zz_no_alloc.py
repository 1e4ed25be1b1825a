"""The allocation-free block-Jacobi entry point (library-owned scratch) matches the workspace one.

It serves callers that cannot pass a workspace or allocate device memory themselves.  The test
calls it on four batches (FP32 GRAM at block width 32, FP32 DIRECT at block width 16, FP64 GRAM),
twice in a row on each (the fixed scratch keeps the previous call's contents), and compares every
result with batched_svd_block_jacobi on a torch-allocated workspace, within the tolerance of the
other block-tier tests (1e-5 FP32, 1e-12 FP64).  It also checks that a batch
needing more than the fixed scratch is refused before any launch.
"""
import numpy as np
import pytest

import gen

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bs():
    import paper_1707_05141_gb300 as bs
    bs.build()
    assert torch.cuda.is_available()
    return bs


def _alloc(bs, a, m, n):
    bsz = a.shape[0]
    k = min(m, n)
    dev = a.device
    s = torch.full((bsz, 1, k), float("nan"), device=dev, dtype=a.dtype)
    u = torch.full((bsz, k, m), float("nan"), device=dev, dtype=a.dtype)
    v = torch.full((bsz, k, n), float("nan"), device=dev, dtype=a.dtype)
    info = torch.zeros(bsz, dtype=torch.int32, device=dev)
    return (bs.Batch.uniform(a, m, n), bs.Batch.uniform(s, k, 1), bs.Batch.uniform(u, m, k),
            bs.Batch.uniform(v, n, k), info, (s, u, v))


def _reference(bs, a, m, n, bw, method):
    A, S, U, V, info, outs = _alloc(bs, a, m, n)
    ws = torch.empty(bs.batched_svd_block_jacobi_workspace(A, bw, method), dtype=torch.uint8, device=a.device)
    bs.batched_svd_block_jacobi(A, S, U, V, info, ws, block_width=bw, method=method)
    return outs, info


def _noalloc(bs, a, m, n, bw, method):
    A, S, U, V, info, outs = _alloc(bs, a, m, n)
    bs.batched_svd_block_jacobi_noalloc(A, S, U, V, info, block_width=bw, method=method)
    return outs, info


# (workload tag, batch, m, n, dtype, block width, method, spectrum): FP32 GRAM with the tensor-core
# Gram, FP32 DIRECT with block width 16 (the pair QR's packed buffers are laid out differently in
# the scratch), and FP64 GRAM (FP64 SIMT products)
CASES = [
    (71, 12, 256, 200, np.float32, 32, 0, lambda i: np.logspace(0, -4, 200)),
    (72, 20, 160, 160, np.float32, 32, 0, lambda i: np.exp(-np.arange(160) / 16.0)),
    (73, 9, 192, 130, np.float32, 16, 1, lambda i: np.logspace(0, -3, 130)),
    (74, 6, 128, 96, np.float64, 32, 0, lambda i: np.logspace(0, -6, 96)),
]


def test_noalloc_matches_workspace_entry_point_twice(bs):
    for tag, nb, m, n, dt, bw, method, sig in CASES:   # consecutive calls share the fixed scratch
        b = gen.uniform_batch(tag, nb, m, n, dt, sig)
        a = torch.from_numpy(b.a).cuda()
        g = 1e-5 if dt == np.float32 else 1e-12
        for call in range(2):                           # two calls in a row on the same batch
            (s0, u0, v0), i0 = _reference(bs, a, b.m, b.n, bw, method)
            (s1, u1, v1), i1 = _noalloc(bs, a, b.m, b.n, bw, method)
            torch.cuda.synchronize()
            assert torch.all(i1 > 0) and torch.all(i1 < (1 << 20)) and torch.equal(i0, i1), (tag, call)
            scale = float(s0.abs().max())
            assert float((s1 - s0).abs().max()) <= g * scale, (tag, call)
            assert float((u1 - u0).abs().max()) <= g and float((v1 - v0).abs().max()) <= g, (tag, call)
            sig_t = torch.from_numpy(b.sigma).cuda().to(s1.dtype)
            assert float((sig_t - s1.view(b.batch, -1)).abs().max()) <= (1e-5 if dt == np.float32 else 1e-11) * scale


def test_noalloc_refuses_batches_beyond_its_scratch(bs):
    dev = torch.device("cuda")
    a = torch.zeros((400, 512, 512), device=dev)          # needs about 100 MiB of scratch
    A, S, U, V, info, _ = _alloc(bs, a, 512, 512)
    assert bs.batched_svd_block_jacobi_workspace(A, 32, bs.BLOCK_GRAM) > bs.NOALLOC_SCRATCH_BYTES
    info.fill_(-7)
    with pytest.raises(bs.BsvdError) as e:
        bs.batched_svd_block_jacobi_noalloc(A, S, U, V, info, block_width=32)
    assert e.value.code == bs.ERR_SCRATCH_LIMIT
    torch.cuda.synchronize()
    assert int(info.min()) == -7 and int(info.max()) == -7      # nothing was launched
