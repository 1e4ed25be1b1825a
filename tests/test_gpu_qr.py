"""GPU parity: batched Householder QR (Algorithm 1) through the C ABI vs the FP64 oracle."""
import numpy as np
import pytest

import gen
import oracle as O
from parity import gate, qr_errors, unit

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bs():
    import paper_1707_05141_gb300 as bs
    bs.build()
    assert torch.cuda.is_available()
    return bs


def _host(t):
    return t.detach().cpu().numpy().astype(np.float64)


def _check_uniform(bs, batch_obj, idx, dtype):
    dev = torch.device("cuda")
    a = torch.from_numpy(batch_obj.a).to(dev)
    q, r, info = bs.qr(a)
    torch.cuda.synchronize()
    assert np.all(info.cpu().numpy() == 0)
    mats = [batch_obj.a64(i) for i in idx]
    Qo, Ro, _ = O.qr_batch(mats)
    qh, rh = _host(q), _host(r)
    u = unit(dtype)
    for j, i in enumerate(idx):
        e = qr_errors(mats[j], qh[i].T, rh[i].T, Qo[j], Ro[j], dtype)
        assert e["r"] <= 1.0 and e["q"] <= 1.0, (i, e)
        assert e["tril_zero"]
        assert e["orth_q"] <= gate(dtype) and e["resid"] <= gate(dtype), (i, e)


def test_qr_fp64_32x32_full_batch(bs):
    """1000 FP64 32 x 32 matrices, sigma_i = 10^(-8 i/31): every matrix against the oracle."""
    b = gen.fp64_32_graded(batch=1000)
    _check_uniform(bs, b, range(1000), np.float64)


def test_qr_fp32_128x32_full_batch_sampled(bs):
    """20000 FP32 128 x 32 matrices in one launch; 96 sampled matrices checked."""
    b = gen.qr128x32_exp8(batch=20000)
    idx = list(range(0, 20000, 20000 // 64))[:64] + list(range(19968, 20000))
    _check_uniform(bs, b, idx, np.float32)


RAGGED = [(1, 1), (2, 1), (7, 3), (33, 33), (64, 1), (100, 37), (129, 64), (5, 0), (0, 0), (31, 31), (48, 17),
          (256, 96)]


# the warp-per-matrix register form: FP32 m <= 128, n <= 32 (one column per lane) and m <= 64,
# n <= 64 (two); FP64 m <= 64, n <= 32
WARP_F32 = [(1, 1), (2, 1), (7, 3), (33, 32), (64, 1), (100, 31), (128, 32), (5, 0), (0, 0), (31, 31), (48, 17),
            (127, 32)]
WARP_F32_WIDE = [(64, 64), (63, 40), (33, 33), (64, 33), (2, 2), (60, 59), (0, 0), (40, 1)]
# tall and wide FP32 panels (the randomized SVD's 256 x l samples): the CTA kernel with 512 threads,
# every matrix of the batch in it, the small ones included
TALL_F32 = [(256, 160), (255, 129), (200, 97), (129, 65), (256, 66), (130, 2), (3, 1), (0, 0), (64, 64), (160, 33),
          (33, 0)]
WARP_F64 = [(1, 1), (64, 32), (37, 20), (40, 32), (64, 1), (50, 31), (3, 0), (32, 32), (2, 2), (63, 31)]


@pytest.mark.parametrize("dt,shapes,special", [
    (np.float32, RAGGED, (3, 5)), (np.float64, RAGGED, (3, 5)),
    (np.float32, WARP_F32, (3, 5)), (np.float32, WARP_F32_WIDE, (0, 1)), (np.float64, WARP_F64, (1, 5)),
    (np.float32, TALL_F32, (0, 2)),
    (np.float32, [(256, 192), (255, 191), (3, 2)], ()),    # 200 KiB in shared memory
    (np.float32, [(1024, 16), (1000, 15), (17, 16)], ()),  # tallest supported
    (np.float64, [(1024, 24), (512, 20)], ())])
def test_qr_ragged_shapes_and_edges(bs, dt, shapes, special):
    rng = np.random.default_rng(7)
    mats = [rng.standard_normal(sh) * 10.0 ** rng.uniform(-2, 2) for sh in shapes]
    if special:
        z, rep = special
        mats[z][:, 5] = 0.0                  # a zero column: identity reflector
        mats[rep][:, 10] = mats[rep][:, 2]  # repeated column: R is rank deficient
    special = set(special)
    ms = np.array([s[0] for s in shapes], np.int32)
    ns = np.array([s[1] for s in shapes], np.int32)
    sizes = (ms.astype(np.int64) * ns + 1)
    off = np.concatenate([[0], np.cumsum(sizes)[:-1]])
    flat = np.zeros(int(sizes.sum()), dt)
    for a, o in zip(mats, off):
        flat[o:o + a.size] = a.T.reshape(-1).astype(dt)
    offq = off.copy()
    r_sizes = ns.astype(np.int64) ** 2 + 1
    offr = np.concatenate([[0], np.cumsum(r_sizes)[:-1]])
    dev = torch.device("cuda")
    fa = torch.from_numpy(flat).to(dev)
    fq = torch.full_like(fa, float("nan"))
    fr = torch.full((int(r_sizes.sum()),), float("nan"), dtype=fa.dtype, device=dev)
    A = bs.Batch.packed(fa, off, ms, ns)
    Q = bs.Batch.packed(fq, offq, ms, ns)
    R = bs.Batch.packed(fr, offr, ns, ns)
    info = torch.empty(len(shapes), dtype=torch.int32, device=dev)
    bs.batched_qr(A, Q, R, info)
    torch.cuda.synchronize()
    assert np.all(info.cpu().numpy() == 0)
    fqh, frh = fq.cpu().numpy().astype(np.float64), fr.cpu().numpy().astype(np.float64)
    for b, ((m, n), a) in enumerate(zip(shapes, mats)):
        if n == 0:
            continue
        a64 = flat[off[b]:off[b] + m * n].reshape(n, m).T.astype(np.float64)
        qg = fqh[offq[b]:offq[b] + m * n].reshape(n, m).T
        rg = frh[offr[b]:offr[b] + n * n].reshape(n, n).T
        qo, ro = O.qr(a64)
        e = qr_errors(a64, qg, rg, qo, ro, dt)
        assert e["tril_zero"], (shapes[b], e)
        if b not in special:                 # rank deficient: trailing rows of R are not unique
            assert e["r"] <= 1.0, (shapes[b], e)
        assert e["orth_q"] <= gate(dt), (shapes[b], e)
        assert e["resid"] <= gate(dt), (shapes[b], e)
        if "q" in e and b not in special:   # rank-deficient cases: Q not unique
            assert e["q"] <= 1.0, (shapes[b], e)


def test_qr_bad_shapes_flagged_and_neighbours_intact(bs):
    dev = torch.device("cuda")
    shapes = [(4, 6), (8, 4), (3, 3)]            # m < n is invalid for QR
    ms = np.array([s[0] for s in shapes], np.int32)
    ns = np.array([s[1] for s in shapes], np.int32)
    off = np.array([0, 64, 128])
    rng = np.random.default_rng(0)
    flat = rng.standard_normal(192).astype(np.float32)
    fa = torch.from_numpy(flat).to(dev)
    fq = torch.zeros_like(fa)
    fr = torch.zeros(192, dtype=torch.float32, device=dev)
    info = torch.empty(3, dtype=torch.int32, device=dev)
    bs.batched_qr(bs.Batch.packed(fa, off, ms, ns), bs.Batch.packed(fq, off, ms, ns),
                  bs.Batch.packed(fr, off, ns, ns), info)
    torch.cuda.synchronize()
    inf = info.cpu().numpy()
    assert inf[0] == bs.INFO_BAD_SHAPE and inf[1] == 0 and inf[2] == 0
    assert np.all(fq.cpu().numpy()[:24] == 0)  # the invalid matrix's outputs untouched


def test_qr_host_argument_errors(bs):
    dev = torch.device("cuda")
    a = torch.zeros((2, 4, 8), device=dev)
    A = bs.Batch.uniform(a, 8, 4)
    info = torch.empty(2, dtype=torch.int32, device=dev)
    L = bs.lib()
    assert L.batched_qr(7, 2, 8, 4, None, None, None, None, None, None, None, None, None, None) == -1
    assert L.batched_qr(0, -1, 8, 4, None, None, None, None, None, None, None, None, None, None) == -2
    assert L.batched_qr(0, 2, 8, 4, None, None, None, None, None, None, None, None, None, None) == -5
    with pytest.raises(bs.BsvdError):
        bs.batched_qr(A, None, None, None)           # d_info missing -> argument 13
    assert bs.lib().batched_qr(0, 2, 8, 9, A.ptrs.data_ptr(), A.m.data_ptr(), A.n.data_ptr(), A.ld.data_ptr(),
                               None, None, None, None, info.data_ptr(), None) == -4
    assert bs.lib().batched_qr(0, 2, 2048, 4, A.ptrs.data_ptr(), A.m.data_ptr(), A.n.data_ptr(), A.ld.data_ptr(),
                               None, None, None, None, info.data_ptr(), None) == bs.ERR_UNSUPPORTED
    assert bs.lib().batched_qr(0, 0, 8, 4, None, None, None, None, None, None, None, None, None, None) == 0


def test_qr_r_only_and_q_only(bs):
    b = gen.qr128x32_exp8(batch=16)
    dev = torch.device("cuda")
    a = torch.from_numpy(b.a).to(dev)
    q1, r1, _ = bs.qr(a)
    _, r2, _ = bs.qr(a, want_q=False)
    q3, _, _ = bs.qr(a, want_r=False)
    torch.cuda.synchronize()
    assert torch.equal(r1, r2) and torch.equal(q1, q3)


# ---- blocked QR (32-column panels, compact WY trailing updates) for matrices beyond the
# shared-memory kernel: tall panels past 1024 rows and large squares (Sections 3.1-3.2) ----

BLOCKED = [(np.float32, 1533, 96, 3, lambda i: np.logspace(0, -3, 96)),      # the tallest panel on chip
           (np.float32, 1200, 300, 2, lambda i: np.exp(-np.arange(300) / 40.0)),
           (np.float32, 700, 700, 2, lambda i: np.logspace(0, -4, 700)),      # a large square, 22 panels
           (np.float64, 733, 200, 2, lambda i: np.logspace(0, -8, 200)),
           (np.float64, 500, 500, 2, lambda i: 10.0 ** (-8.0 * np.arange(500) / 499)),
           # panels taller than one CTA's shared memory: a cluster of CTAs per panel
           (np.float32, 4096, 96, 2, lambda i: np.logspace(0, -3, 96)),             # 3 CTAs
           (np.float32, 11976, 40, 1, lambda i: np.logspace(0, -2, 40)),            # the tallest: 8 CTAs (*)
           (np.float32, 2000, 600, 1, lambda i: np.exp(-np.arange(600) / 80.0)),    # 2 CTAs, 19 panels
           (np.float64, 5576, 48, 1, lambda i: np.logspace(0, -8, 48)),             # 8 CTAs
           (np.float64, 1500, 300, 1, lambda i: 10.0 ** (-6.0 * np.arange(300) / 299))]


@pytest.mark.parametrize("dt,m,n,nb,sig", BLOCKED)
def test_qr_blocked_against_oracle(bs, dt, m, n, nb, sig):
    """Every matrix of the batch against the oracle's Householder QR: R and Q after sign alignment,
    exact zeros below R's diagonal, orthogonality and residual at the gate.  (*) The oracle forms
    the full m x m Q, out of reach at 11 976 rows: there the properties that hold at any size are
    checked (R's diagonal magnitudes against the generator's spectrum's bounds included)."""
    b = gen.uniform_batch(81, nb, m, n, dt, sig)
    a = torch.from_numpy(b.a).cuda()
    q, r, info = bs.qr_blocked(a)
    torch.cuda.synchronize()
    assert np.all(info.cpu().numpy() == 0)
    if m > 8000:
        qh, rh = _host(q), _host(r)
        for i in range(nb):
            a64, qq, rr = b.a64(i), qh[i].T, rh[i].T
            assert np.all(np.tril(rr, -1) == 0.0)
            assert np.abs(qq.T @ qq - np.eye(n)).max() <= gate(dt)
            assert np.linalg.norm(a64 - qq @ rr) / np.linalg.norm(a64) <= gate(dt)
            # |det R| = prod sigma: the R factor carries A's volume
            assert abs(np.sum(np.log(np.abs(np.diag(rr)))) - np.sum(np.log(b.sigma[i]))) <= 1e-3
        return
    mats = [b.a64(i) for i in range(nb)]
    Qo, Ro, _ = O.qr_batch(mats)
    qh, rh = _host(q), _host(r)
    for i in range(nb):
        e = qr_errors(mats[i], qh[i].T, rh[i].T, Qo[i], Ro[i], dt)
        assert e["r"] <= 1.0 and e["q"] <= 1.0, (i, e)
        assert e["tril_zero"]
        assert e["orth_q"] <= gate(dt) and e["resid"] <= gate(dt), (i, e)


def test_qr_blocked_ragged_and_bad_shapes(bs):
    """A ragged FP32 batch (1 x 1, single columns, n = 0, a panel edge at 32 and 33 columns, the
    tallest height) with one wide matrix, which is flagged and left untouched; Q-only and R-only
    calls give the same factors."""
    shapes = [(1533, 40), (1, 1), (64, 64), (100, 1), (5, 0), (300, 299), (1000, 33), (129, 32), (40, 60)]
    rng = np.random.default_rng(3)
    mats = [rng.standard_normal((m, n)) for m, n in shapes]
    dev = torch.device("cuda")
    ms = np.array([s[0] for s in shapes], np.int32)
    ns = np.array([s[1] for s in shapes], np.int32)
    ks = np.minimum(ms, ns)
    offA = np.concatenate([[0], np.cumsum(ms.astype(np.int64) * ns + 1)[:-1]])
    offR = np.concatenate([[0], np.cumsum(ns.astype(np.int64) * ns + 1)[:-1]])
    flat = np.zeros(int(offA[-1] + ms[-1] * ns[-1] + 1), np.float32)
    for mat, o in zip(mats, offA):
        flat[o:o + mat.size] = mat.T.reshape(-1)
    fa = torch.from_numpy(flat).to(dev)
    results = []
    for want_q, want_r in ((True, True), (True, False), (False, True)):
        fq = torch.full_like(fa, float("nan"))
        fr = torch.full((int(offR[-1] + ns[-1] ** 2 + 1),), float("nan"), device=dev)
        info = torch.full((len(shapes),), -7, dtype=torch.int32, device=dev)
        A = bs.Batch.packed(fa, offA, ms, ns)
        ws = torch.empty(bs.batched_qr_blocked_workspace(A), dtype=torch.uint8, device=dev)
        bs.batched_qr_blocked(A, bs.Batch.packed(fq, offA, ms, ns) if want_q else None,
                              bs.Batch.packed(fr, offR, ns, ns) if want_r else None, info, ws)
        torch.cuda.synchronize()
        results.append((fq.cpu().numpy().astype(np.float64), fr.cpu().numpy().astype(np.float64), info.cpu().numpy()))
    fq, fr, info = results[0]
    assert all(np.array_equal(r[2], info) for r in results)
    assert np.array_equal(results[1][0], fq, equal_nan=True) and np.array_equal(results[2][1], fr, equal_nan=True)
    assert np.all(np.isnan(results[1][1])) and np.all(np.isnan(results[2][0]))
    for b, ((m, n), mat) in enumerate(zip(shapes, mats)):
        if m < n:
            assert info[b] == bs.INFO_BAD_SHAPE
            assert np.all(np.isnan(fq[offA[b]:offA[b] + m * n])) and np.all(np.isnan(fr[offR[b]:offR[b] + n * n]))
            continue
        assert info[b] == 0, (m, n, info[b])
        if n == 0:
            continue
        a64 = flat[offA[b]:offA[b] + m * n].reshape(n, m).T.astype(np.float64)
        qo, ro = O.qr(a64)
        q = fq[offA[b]:offA[b] + m * n].reshape(n, m).T
        r = fr[offR[b]:offR[b] + n * n].reshape(n, n).T
        e = qr_errors(a64, q, r, qo, ro, np.float32)
        assert e["r"] <= 1.0 and e["q"] <= 1.0 and e["tril_zero"], ((m, n), e)
        assert e["orth_q"] <= 1e-5 and e["resid"] <= 1e-5, ((m, n), e)


def test_qr_blocked_agrees_with_the_shared_memory_kernel(bs):
    """On shapes both kernels take, the blocked QR and the one-CTA kernel give the same factors
    within rounding (the same reflectors, applied in another order)."""
    b = gen.uniform_batch(82, 64, 256, 96, np.float32, lambda i: np.exp(-np.arange(96) / 16.0))
    a = torch.from_numpy(b.a).cuda()
    q0, r0, i0 = bs.qr(a)
    q1, r1, i1 = bs.qr_blocked(a)
    torch.cuda.synchronize()
    assert torch.equal(i0, i1)
    scale = float(r0.abs().max())
    assert float((r1 - r0).abs().max()) <= 64 * 6e-8 * 16 * scale
    assert float((q1 - q0).abs().max()) <= 1e-4


def test_qr_blocked_cluster_panels_ragged(bs):
    """Tall and short matrices in one batch whose bound needs the cluster panels: every matrix
    against the oracle (the short ones factored by the same cluster launch)."""
    shapes = [(3000, 33), (40, 40), (1600, 1), (12, 5), (2500, 70), (33, 32)]
    rng = np.random.default_rng(8)
    mats = [rng.standard_normal((m, n)) * np.logspace(0, -2, n) for m, n in shapes]
    dev = torch.device("cuda")
    ms = np.array([s[0] for s in shapes], np.int32)
    ns = np.array([s[1] for s in shapes], np.int32)
    offA = np.concatenate([[0], np.cumsum(ms.astype(np.int64) * ns + 1)[:-1]])
    offR = np.concatenate([[0], np.cumsum(ns.astype(np.int64) * ns + 1)[:-1]])
    flat = np.zeros(int(offA[-1] + ms[-1] * ns[-1] + 1), np.float32)
    for mat, o in zip(mats, offA):
        flat[o:o + mat.size] = mat.T.reshape(-1)
    fa = torch.from_numpy(flat).to(dev)
    fq = torch.full_like(fa, float("nan"))
    fr = torch.full((int(offR[-1] + ns[-1] ** 2 + 1),), float("nan"), device=dev)
    info = torch.full((len(shapes),), -7, dtype=torch.int32, device=dev)
    A = bs.Batch.packed(fa, offA, ms, ns)
    ws = torch.empty(bs.batched_qr_blocked_workspace(A), dtype=torch.uint8, device=dev)
    bs.batched_qr_blocked(A, bs.Batch.packed(fq, offA, ms, ns), bs.Batch.packed(fr, offR, ns, ns), info, ws)
    torch.cuda.synchronize()
    fq, fr, info = fq.cpu().numpy().astype(np.float64), fr.cpu().numpy().astype(np.float64), info.cpu().numpy()
    for b, (m, n) in enumerate(shapes):
        assert info[b] == 0, (m, n, info[b])
        a64 = flat[offA[b]:offA[b] + m * n].reshape(n, m).T.astype(np.float64)
        qo, ro = O.qr(a64)
        q = fq[offA[b]:offA[b] + m * n].reshape(n, m).T
        r = fr[offR[b]:offR[b] + n * n].reshape(n, n).T
        e = qr_errors(a64, q, r, qo, ro, np.float32)
        assert e["r"] <= 1.0 and e["q"] <= 1.0 and e["tril_zero"], ((m, n), e)
        assert e["orth_q"] <= 1e-5 and e["resid"] <= 1e-5, ((m, n), e)
