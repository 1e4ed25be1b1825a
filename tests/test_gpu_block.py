"""GPU parity: batched one-sided block Jacobi (Algorithm 3) through the C ABI vs the FP64 oracle."""
import numpy as np
import pytest

import gen
import oracle as O
from parity import gate, svd_errors

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bs():
    import paper_1707_05141_gb300 as bs
    bs.build()
    assert torch.cuda.is_available()
    return bs


def _host(*ts):
    return [t.detach().cpu().numpy().astype(np.float64) for t in ts]


@pytest.fixture(scope="module")
def w2():
    """Four 512 x 512 FP32 matrices with sigma log-uniform on [1e-6, 1] and their oracle SVDs."""
    b = gen.block512_loguniform(batch=4)
    mats = [b.a64(i) for i in range(b.batch)]
    Uo, So, Vo, info, _ = O.svd_batch(mats)
    return b, mats, So


QR = 1 << 18   # BSVD_BLOCK_QR_PRECONDITION


@pytest.mark.parametrize("method,bw", [(0, 32), (1, 32), (0, 16), (1, 16), (0 | (1 << 16), 32), (0 | QR, 32),
                                       (1 | QR, 32), (0 | QR, 16)])
def test_block_512_log_uniform_sigma(bs, w2, method, bw):
    """FP32 with bw = 32 forms the pair Gram matrices on the tensor cores; the BLOCK_SIMT_PRODUCTS
    flag keeps them on the SIMT pipes; BLOCK_QR_PRECONDITION runs the block Jacobi on R^T of a
    blocked Householder QR and forms U = Q V~ (about half the outer sweeps)."""
    b, mats, So = w2
    a = torch.from_numpy(b.a).cuda()
    u, s, v, info, rots = bs.svd_block(a, block_width=bw, method=method, max_sweeps=30)
    torch.cuda.synchronize()
    if method & QR:      # fewer outer sweeps than on A itself (14-15 on these matrices)
        assert int(info.cpu().numpy().max()) <= 11, info.cpu().numpy()
    method &= 0xff
    u, s, v = _host(u, s, v)
    info = info.cpu().numpy()
    for i in range(b.batch):
        assert 0 < info[i] < (1 << 20), (i, info[i])
        e = svd_errors(mats[i], u[i].T, s[i], v[i].T, So[i])
        # every gate at 1e-5, U's orthogonality over all columns down to sigma = 1e-6 (DIRECT: its
        # pair threshold 4 sqrt(512) u = 5.4e-6 bounds the cosines left between columns)
        assert max(e.values()) <= 1e-5, (i, method, e)


@pytest.mark.parametrize("bw", [16, 32])
@pytest.mark.parametrize("dt", [np.float32, np.float64])
@pytest.mark.parametrize("method", [0, 1, 0 | QR, 1 | QR])
def test_block_ragged_shapes(bs, dt, method, bw):
    """Partial last block, a virtual empty block, wide input, tiny block counts."""
    shapes = [(96, 80), (70, 130), (64, 64), (200, 33), (33, 33), (5, 3)]
    rng = np.random.default_rng(21)
    g = gate(dt)
    for (m, n) in shapes:
        k = min(m, n)
        uu, _ = np.linalg.qr(rng.standard_normal((m, k)))
        vv, _ = np.linalg.qr(rng.standard_normal((n, k)))
        sig = np.sort(10.0 ** rng.uniform(-2, 0, k))[::-1]
        a64 = (uu * sig) @ vv.T
        a = torch.from_numpy(np.ascontiguousarray(a64.T.astype(dt))[None]).cuda()
        u, s, v, info, rots = bs.svd_block(a, block_width=bw, method=method, max_sweeps=30)
        torch.cuda.synchronize()
        u, s, v = _host(u, s, v)
        assert 0 < int(info[0]) < (1 << 20), ((m, n), int(info[0]))
        ad = a64.astype(dt).astype(np.float64)
        _, so, _, _, _ = O.svd(ad)
        e = svd_errors(ad, u[0].T, s[0], v[0].T, so)
        assert max(e.values()) <= g, ((m, n), e)


@pytest.mark.parametrize("method", [0, 1 << 16])
def test_block_packed_uneven_batch(bs, method):
    """One call over matrices of different shapes and odd leading dimensions (the tensor-core
    Gram's scalar-load path and partial 32-row chunks), FP32, bw = 32."""
    shapes = [(300, 200), (130, 257), (64, 64), (211, 97), (257, 300), (40, 190)]
    rng = np.random.default_rng(5)
    mats, offs, lds, o = [], [], [], 0
    for (m, n) in shapes:
        k = min(m, n)
        uu, _ = np.linalg.qr(rng.standard_normal((m, k)))
        vv, _ = np.linalg.qr(rng.standard_normal((n, k)))
        sig = np.sort(10.0 ** rng.uniform(-4, 0, k))[::-1]
        a64 = ((uu * sig) @ vv.T).astype(np.float32).astype(np.float64)
        ld = m + 3                                   # not a multiple of 4
        mats.append(a64)
        offs.append(o)
        lds.append(ld)
        o += ld * n
    flat = np.zeros(o, np.float32)
    for a64, off, ld in zip(mats, offs, lds):
        m, n = a64.shape
        buf = np.zeros((n, ld), np.float32)
        buf[:, :m] = a64.T
        flat[off:off + ld * n] = buf.reshape(-1)
    dev = torch.device("cuda")
    A = bs.Batch.packed(torch.from_numpy(flat).to(dev), offs, [s[0] for s in shapes], [s[1] for s in shapes], lds)
    ks = [min(s) for s in shapes]
    ou = np.cumsum([0] + [m * k for (m, _), k in zip(shapes, ks)])
    ov = np.cumsum([0] + [n * k for (_, n), k in zip(shapes, ks)])
    oks = np.cumsum([0] + ks)
    U = torch.zeros(int(ou[-1]), device=dev)
    V = torch.zeros(int(ov[-1]), device=dev)
    S = torch.zeros(int(oks[-1]), device=dev)
    Ub = bs.Batch.packed(U, ou[:-1], [s[0] for s in shapes], ks)
    Vb = bs.Batch.packed(V, ov[:-1], [s[1] for s in shapes], ks)
    Sb = bs.Batch.packed(S, oks[:-1], ks, [1] * len(ks))
    info = torch.zeros(len(shapes), dtype=torch.int32, device=dev)
    ws = torch.empty(bs.batched_svd_block_jacobi_workspace(A, 32, method), dtype=torch.uint8, device=dev)
    bs.batched_svd_block_jacobi(A, Sb, Ub, Vb, info, ws, block_width=32, method=method, max_sweeps=30)
    torch.cuda.synchronize()
    Uh, Vh, Sh = (t.cpu().numpy().astype(np.float64) for t in (U, V, S))
    for i, ((m, n), k) in enumerate(zip(shapes, ks)):
        assert 0 < int(info[i]) < (1 << 20), (i, int(info[i]))
        u = Uh[ou[i]:ou[i + 1]].reshape(k, m).T
        v = Vh[ov[i]:ov[i + 1]].reshape(k, n).T
        _, so, _, _, _ = O.svd(mats[i])
        e = svd_errors(mats[i], u, Sh[oks[i]:oks[i + 1]], v, so)
        assert max(e.values()) <= 1e-5, ((m, n), e)


def test_block_matches_register_tier_on_64x64(bs):
    b = gen.svd64_exp8(batch=32)
    a = torch.from_numpy(b.a).cuda()
    _, s_reg, _, _, _ = bs.svd(a)
    _, s_blk, _, info, _ = bs.svd_block(a, block_width=16, method=0)
    torch.cuda.synchronize()
    assert torch.all(info > 0)
    assert (s_reg - s_blk).abs().max().item() <= 2e-6


def test_block_workspace_and_errors(bs):
    dev = torch.device("cuda")
    a = torch.zeros((2, 40, 40), device=dev)
    A = bs.Batch.uniform(a, 40, 40)
    need = bs.batched_svd_block_jacobi_workspace(A, 16, 0)
    assert need > 0
    s = torch.zeros((2, 1, 40), device=dev)
    u = torch.zeros((2, 40, 40), device=dev)
    v = torch.zeros((2, 40, 40), device=dev)
    info = torch.zeros(2, dtype=torch.int32, device=dev)
    small = torch.empty(need - 1, dtype=torch.uint8, device=dev)
    with pytest.raises(bs.BsvdError) as e:
        bs.batched_svd_block_jacobi(A, bs.Batch.uniform(s, 40, 1), bs.Batch.uniform(u, 40, 40),
                                    bs.Batch.uniform(v, 40, 40), info, small, block_width=16)
    assert e.value.code == bs.ERR_WORKSPACE
    ws = torch.empty(need, dtype=torch.uint8, device=dev)
    with pytest.raises(bs.BsvdError) as e:
        bs.batched_svd_block_jacobi(A, bs.Batch.uniform(s, 40, 1), bs.Batch.uniform(u, 40, 40),
                                    bs.Batch.uniform(v, 40, 40), info, ws, block_width=24)
    assert e.value.code == -16
    # a zero matrix converges in one sweep with zero singular values
    bs.batched_svd_block_jacobi(A, bs.Batch.uniform(s, 40, 1), bs.Batch.uniform(u, 40, 40),
                                bs.Batch.uniform(v, 40, 40), info, ws, block_width=16)
    torch.cuda.synchronize()
    assert info.tolist() == [1, 1] and float(s.abs().max()) == 0.0


RETEST = 1 << 19   # BSVD_BLOCK_RETEST_ALL


def _bits(t):
    return t.view(torch.int32) if t.dtype == torch.float32 else t.view(torch.int64)


@pytest.mark.parametrize("method,bw,dt", [(0, 32, np.float32), (0 | (1 << 16), 32, np.float32), (1, 32, np.float32),
                                          (0 | QR, 32, np.float32), (0, 16, np.float64), (1 | QR, 16, np.float64)])
def test_block_pair_selection_is_exact(bs, method, bw, dt):
    """Pairs found orthogonal are not tested again while their blocks are unchanged (adaptive pair
    selection, Section 6.3); the skipped tests would have come out the same, so U, S, V, the sweep
    counts and the rotation counts equal those of re-testing every pair, bit for bit."""
    b = gen.uniform_batch(91, 6, 320, 256, dt, lambda i: np.logspace(0, -5 if dt == np.float32 else -9, 256))
    a = torch.from_numpy(b.a).cuda()
    r0 = bs.svd_block(a, block_width=bw, method=method | RETEST, max_sweeps=30)
    r1 = bs.svd_block(a, block_width=bw, method=method, max_sweeps=30)
    torch.cuda.synchronize()
    for x, y in zip(r0[:3], r1[:3]):
        assert torch.equal(_bits(x), _bits(y)), method
    assert torch.equal(r0[3], r1[3]) and torch.equal(r0[4], r1[4]), method
    info = r1[3].cpu().numpy()
    assert np.all((info > 0) & (info < (1 << 20))), info


def test_block_qr_preconditioning_on_tall_matrices(bs):
    """The block tier on R^T of a blocked QR whose panels (2600 rows) need a cluster of CTAs each:
    sigma, orthogonality and residual against the oracle at the FP32 gate."""
    b = gen.uniform_batch(92, 2, 2600, 96, np.float32, lambda i: np.logspace(0, -4, 96))
    a = torch.from_numpy(b.a).cuda()
    u, s, v, info, rots = bs.svd_block(a, block_width=32, method=QR, max_sweeps=30)
    torch.cuda.synchronize()
    u, s, v = _host(u, s, v)
    info = info.cpu().numpy()
    for i in range(b.batch):
        assert 0 < info[i] < (1 << 20), (i, info[i])
        a64 = b.a64(i)
        So = O.svd(a64)[1]
        e = svd_errors(a64, u[i].T, s[i], v[i].T, So)
        assert max(e.values()) <= 1e-5, (i, e)


def test_block_width_autotuned(bs, tmp_path, monkeypatch):
    """The autotuner times both block widths (and, for GRAM, the inner register variant) and records
    the fastest; block_width = 0 then runs that choice: the same result bit for bit as naming it."""
    from paper_1707_05141_gb300 import autotune
    monkeypatch.setattr(autotune, "CACHE", str(tmp_path / "autotune.json"))
    b = gen.uniform_batch(93, 8, 256, 256, np.float32, lambda i: np.logspace(0, -4, 256))
    a = torch.from_numpy(b.a).cuda()
    rec = autotune.tune_block(a, method=QR, force=True)
    try:
        assert rec["block_width"] in (16, 32) and len(rec["all_ms"]) == 6
        r0 = bs.svd_block(a, block_width=0, method=QR, max_sweeps=30)
        r1 = bs.svd_block(a, block_width=rec["block_width"], method=QR | (rec["inner_variant"] << 8),
                          max_sweeps=30)
        torch.cuda.synchronize()
        for x, y in zip(r0[:3], r1[:3]):
            assert torch.equal(_bits(x), _bits(y))
        assert torch.equal(r0[3], r1[3])
        assert autotune.tune_block(a, method=QR)["block_width"] == rec["block_width"]   # from the cache
    finally:
        bs.set_block_choice(bs.F32, 256, 256, 0)


def test_block_512_plain_inner_variant(bs, w2):
    """GRAM with the inner 64 x 64 SVDs on the plain carried-norm register variant (X = its V, no
    QR of G; the autotuner's choice on this GPU), on R^T of the blocked QR: every gate at 1e-5."""
    b, mats, So = w2
    k = next(k for k in range(1, bs.jacobi_variants(bs.F32, 64, 64, bs.TIER_REGISTER) + 1)
             if bs.jacobi_variant_desc(bs.F32, 64, 64, k)["carried_norms"]
             and not bs.jacobi_variant_desc(bs.F32, 64, 64, k)["qr_precond"])
    a = torch.from_numpy(b.a).cuda()
    u, s, v, info, rots = bs.svd_block(a, block_width=32, method=QR | (k << 8), max_sweeps=30)
    torch.cuda.synchronize()
    u, s, v = _host(u, s, v)
    info = info.cpu().numpy()
    for i in range(b.batch):
        assert 0 < info[i] < (1 << 20), (i, info[i])
        e = svd_errors(mats[i], u[i].T, s[i], v[i].T, So[i])
        assert max(e.values()) <= 1e-5, (i, e)
