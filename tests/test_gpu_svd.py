"""GPU parity: batched one-sided Jacobi SVD (Algorithm 2) through the C ABI vs the FP64 oracle."""
import os

import numpy as np
import pytest

import gen
import oracle as O
from parity import gate, svd_errors, vector_errors

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bs():
    import paper_1707_05141_gb300 as bs
    bs.build()
    assert torch.cuda.is_available()
    return bs


def _run_uniform(bs, b, **kw):
    dev = torch.device("cuda")
    a = torch.from_numpy(b.a).to(dev)
    u, s, v, info, rots = bs.svd(a, **kw)
    torch.cuda.synchronize()
    return (u.cpu().numpy().astype(np.float64), s.cpu().numpy().astype(np.float64),
            v.cpu().numpy().astype(np.float64), info.cpu().numpy(), rots.cpu().numpy())


def _check(b, idx, u, s, v, info, dtype, vec_c=64.0):
    mats = [b.a64(i) for i in idx]
    Uo, So, Vo, info_o, _ = O.svd_batch(mats)
    g = gate(dtype)
    for j, i in enumerate(idx):
        assert 0 < info[i] < (1 << 20), (i, info[i])
        e = svd_errors(mats[j], u[i].T, s[i], v[i].T, So[j])
        assert max(e.values()) <= g, (i, e)
        assert vector_errors(u[i].T, Uo[j], So[j], dtype, vec_c) <= 1.0, i
        assert vector_errors(v[i].T, Vo[j], So[j], dtype, vec_c) <= 1.0, i
        assert np.all(np.diff(s[i]) <= 0)


def test_svd_fp64_32x32_full_batch(bs):
    """1000 FP64 32 x 32 matrices, kappa = 1e8: every matrix within 1e-12 of the oracle."""
    b = gen.fp64_32_graded(batch=1000)
    u, s, v, info, rots = _run_uniform(bs, b)
    _check(b, range(1000), u, s, v, info, np.float64)
    # the generator's own sigma agrees to the same normwise bound
    assert np.abs(s - b.sigma).max() <= 1e-12


def test_svd_fp32_64x64_full_batch_sampled(bs):
    """20000 FP32 64 x 64 matrices in one launch (the benchmark's launch); 64 sampled + the tail."""
    b = gen.svd64_exp8(batch=20000)
    u, s, v, info, rots = _run_uniform(bs, b)
    idx = list(range(0, 20000, 20000 // 48))[:48] + list(range(19984, 20000))
    _check(b, idx, u, s, v, info, np.float32)
    assert np.all((info > 0) & (info < (1 << 20)))
    assert np.abs(s - b.sigma).max() <= 1e-5


def _packed_case(bs, shapes, dt, seed, mutate=None):
    rng = np.random.default_rng(seed)
    mats = []
    for (m, n) in shapes:
        k = min(m, n)
        if k == 0:
            mats.append(np.zeros((m, n)))
            continue
        uu, _ = np.linalg.qr(rng.standard_normal((m, k)))
        vv, _ = np.linalg.qr(rng.standard_normal((n, k)))
        sig = np.sort(10.0 ** rng.uniform(-3 if dt == np.float64 else -2, 0, k))[::-1]
        mats.append((uu * sig) @ vv.T)
    if mutate:
        mutate(mats)
    ms = np.array([s[0] for s in shapes], np.int32)
    ns = np.array([s[1] for s in shapes], np.int32)
    ks = np.minimum(ms, ns).astype(np.int64)
    def offsets(sz):
        sz = np.asarray(sz, np.int64) + 1
        return np.concatenate([[0], np.cumsum(sz)[:-1]]), int(sz.sum())
    offA, nA = offsets(ms.astype(np.int64) * ns)
    offS, nS = offsets(ks)
    offU, nU = offsets(ms * ks)
    offV, nV = offsets(ns * ks)
    flat = np.zeros(nA, dt)
    for a, o in zip(mats, offA):
        flat[o:o + a.size] = a.T.reshape(-1).astype(dt)
    dev = torch.device("cuda")
    fa = torch.from_numpy(flat).to(dev)
    fs = torch.full((nS,), float("nan"), dtype=fa.dtype, device=dev)
    fu = torch.full((nU,), float("nan"), dtype=fa.dtype, device=dev)
    fv = torch.full((nV,), float("nan"), dtype=fa.dtype, device=dev)
    info = torch.empty(len(shapes), dtype=torch.int32, device=dev)
    rots = torch.empty(len(shapes), dtype=torch.int64, device=dev)
    bs.batched_svd_jacobi(bs.Batch.packed(fa, offA, ms, ns), bs.Batch.packed(fs, offS, ks, np.ones_like(ks)),
                          bs.Batch.packed(fu, offU, ms, ks), bs.Batch.packed(fv, offV, ns, ks), info, rots)
    torch.cuda.synchronize()
    out = []
    fs_h, fu_h, fv_h = (t.cpu().numpy().astype(np.float64) for t in (fs, fu, fv))
    for b, (m, n) in enumerate(shapes):
        k = int(ks[b])
        a64 = flat[offA[b]:offA[b] + m * n].reshape(n, m).T.astype(np.float64)
        out.append((a64, fu_h[offU[b]:offU[b] + m * k].reshape(k, m).T, fs_h[offS[b]:offS[b] + k],
                    fv_h[offV[b]:offV[b] + n * k].reshape(k, n).T))
    return out, info.cpu().numpy(), rots.cpu().numpy()


SHAPES32 = [(1, 1), (2, 2), (3, 2), (2, 5), (17, 17), (33, 31), (31, 64), (64, 64), (65, 7), (128, 128),
            (256, 128), (200, 99), (1, 40), (40, 1), (0, 5), (7, 0)]
SHAPES64 = [(1, 1), (2, 2), (3, 2), (2, 5), (17, 17), (33, 31), (31, 64), (64, 64), (65, 7), (256, 64),
            (200, 33), (1, 40), (40, 1), (0, 3)]


@pytest.mark.parametrize("dt,shapes", [(np.float32, SHAPES32), (np.float64, SHAPES64)])
def test_svd_ragged_shapes(bs, dt, shapes):
    """Ragged batch spanning odd/even n, wide matrices, empty matrices and the tier maximum."""
    res, info, rots = _packed_case(bs, shapes, dt, seed=11)
    g = gate(dt)
    for (m, n), (a64, u, s, v), inf in zip(shapes, res, info):
        k = min(m, n)
        if k == 0:
            assert inf == 0
            continue
        assert 0 < inf < (1 << 20), ((m, n), inf)
        uo, so, vo, _, _ = O.svd(a64)
        e = svd_errors(a64, u, s, v, so)
        assert max(e.values()) <= g, ((m, n), e)
        assert vector_errors(u, uo, so, dt) <= 1.0 and vector_errors(v, vo, so, dt) <= 1.0, (m, n)


def test_svd_degenerate_inputs(bs):
    """Zero matrix, a zero column, repeated singular values, rank one, diagonal input."""
    shapes = [(8, 8), (12, 6), (16, 16), (10, 7), (9, 9)]

    def mutate(mats):
        mats[0][:] = 0.0
        mats[1][:, 3] = 0.0
        q, _ = np.linalg.qr(np.random.default_rng(1).standard_normal((16, 16)))
        mats[2][:] = q * np.array([2.0] * 5 + [1.0] * 11)                 # repeated sigma
        mats[3][:] = np.outer(np.arange(1.0, 11.0), np.linspace(-1, 1, 7))  # rank one
        mats[4][:] = np.diag([3.0, -1.0, 0.5, 7.0, 0.0, 2.0, -2.0, 1.0, 0.25])

    res, info, rots = _packed_case(bs, shapes, np.float64, seed=3, mutate=mutate)
    for (a64, u, s, v), inf, r in zip(res, info, rots):
        so = np.linalg.svd(a64, compute_uv=False)
        assert np.abs(s - so).max() <= 1e-12 * max(so[0], 1.0)
        e = svd_errors(a64, u, s, v, so)
        assert e.get("orth_v", 0) <= 1e-12 and e.get("resid", 0) <= 1e-12, e
        assert np.all(np.isfinite(u)) and np.all(np.isfinite(v))
    a0, u0, s0, v0 = res[0]
    assert np.all(s0 == 0) and np.all(u0 == 0) and info[0] == 1 and rots[0] == 0
    assert rots[4] == 0 and info[4] == 1                      # diagonal: no rotation at all
    assert np.array_equal(res[4][2], np.sort(np.abs(np.diag(res[4][0])))[::-1])


def test_svd_sweep_cap_reports_not_converged(bs):
    b = gen.svd64_exp8(batch=4)
    u, s, v, info, rots = _run_uniform(bs, b, max_sweeps=1)
    assert np.all(info == bs.INFO_NOT_CONVERGED + 1)
    assert np.all(rots > 0) and np.all(rots <= 64 * 63 // 2)


def test_svd_bad_shape_flagged(bs):
    dev = torch.device("cuda")
    a = torch.zeros((3, 8, 8), device=dev)
    A = bs.Batch.uniform(a, 8, 8)
    A.m[1] = 9                        # larger than max_m = 8
    s = torch.zeros((3, 1, 8), device=dev)
    info = torch.empty(3, dtype=torch.int32, device=dev)
    bs.batched_svd_jacobi(A, bs.Batch.uniform(s, 8, 1), None, None, info)
    torch.cuda.synchronize()
    assert list(info.cpu().numpy()) == [1, bs.INFO_BAD_SHAPE, 1]


def test_svd_without_vectors_matches(bs):
    b = gen.svd64_exp8(batch=32)
    dev = torch.device("cuda")
    a = torch.from_numpy(b.a).to(dev)
    u1, s1, v1, i1, r1 = bs.svd(a)
    _, s2, _, i2, r2 = bs.svd(a, want_u=False, want_v=False)
    torch.cuda.synchronize()
    assert torch.equal(s1, s2) and torch.equal(i1, i2) and torch.equal(r1, r2)


def _variant_cases():
    import paper_1707_05141_gb300 as bsm
    cases = []
    for dt, (m, n) in [(np.float32, (64, 64)), (np.float32, (32, 32)), (np.float32, (128, 48)),
                       (np.float32, (40, 100)), (np.float64, (32, 32)), (np.float64, (64, 64)), (np.float64, (64, 60)),
                       (np.float64, (20, 50))]:
        code = 0 if dt == np.float32 else 1
        nv = bsm.jacobi_variants(code, m, n, bsm.TIER_REGISTER) if os.path.exists(bsm.LIB) else 0
        for v in range(1, nv + 1):
            cases.append((dt, m, n, bsm.TIER_REGISTER | (v << 8)))
        cases.append((dt, m, n, bsm.TIER_SHARED))
    return cases


@pytest.mark.parametrize("dt,m,n,tier", _variant_cases())
def test_svd_every_tier_variant(bs, dt, m, n, tier):
    """Each kernel variant the tuner may select: 96 matrices, all against the oracle."""
    k = min(m, n)
    sig = np.exp(-np.arange(k) / 8.0) if dt == np.float32 else 10.0 ** (-8.0 * np.arange(k) / max(k - 1, 1))
    b = gen.uniform_batch(50, 96, m, n, dt, lambda i: sig)
    u, s, v, info, rots = _run_uniform(bs, b, tier=tier)
    _check(b, range(96), u, s, v, info, dt)
