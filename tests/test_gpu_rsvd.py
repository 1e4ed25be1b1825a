"""GPU parity: batched randomized SVD (Algorithm 4 + power step, adaptive range finder) vs the oracle.

The oracle runs the same steps in FP64 with the same Gaussian sampling matrix definition
(Philox4x32-10 from its published definition on both sides) and the number of columns the GPU
reports; the result is also checked against what the mathematics fixes: the truncation error
||A - U_k S_k V_k^T||_F / ||A||_F <= eps, and no rank below the Eckart-Young optimum.
"""
import math

import numpy as np
import pytest

import gen
import oracle as O
from parity import svd_errors, vector_errors

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

EPS = 1e-5
SEED = 20260301


@pytest.fixture(scope="module")
def bs():
    import paper_1707_05141_gb300 as bs
    bs.build()
    assert torch.cuda.is_available()
    return bs


def _unpack(res, b):
    m, n, k = int(res.m[b]), int(res.n[b]), int(res.rank[b])
    fu = res.U_h[res.off_u[b]:res.off_u[b] + m * k].reshape(k, m).T
    fv = res.V_h[res.off_v[b]:res.off_v[b] + n * k].reshape(k, n).T
    fs = res.S_h[res.off_s[b]:res.off_s[b] + k]
    return fu, fs, fv


def _run(bs, rb, hint, **kw):
    flat = torch.from_numpy(rb.flat).cuda()
    res = bs.rsvd(flat, rb.offset, rb.m, rb.n, rank_hint=hint, tol=EPS, seed=SEED, **kw)
    torch.cuda.synchronize()
    res.U_h = res.U.cpu().numpy().astype(np.float64)
    res.V_h = res.V.cpu().numpy().astype(np.float64)
    res.S_h = res.S.cpu().numpy().astype(np.float64)
    res.rank_h = res.rank.cpu().numpy()
    res.info_h = res.info.cpu().numpy()
    res.samples_h = res.samples.cpu().numpy()
    return res


def _check_block(rb, res, b, compare_oracle=True):
    a = rb.a64(b)
    u, s, v = _unpack(res, b)
    na = np.linalg.norm(a)
    err = np.linalg.norm(a - (u * s) @ v.T) / na
    assert err <= EPS, (b, err, int(res.rank_h[b]), int(res.samples_h[b]))
    sv = np.linalg.svd(a, compute_uv=False)
    k_opt = O.trunc_rank(sv, na, EPS)
    assert int(res.rank_h[b]) >= k_opt - 1, (b, int(res.rank_h[b]), k_opt)
    # overshoot above the Eckart-Young optimum comes from the estimate's budget (4 est^2) and the
    # 5% margin; with sigma ratios near 0.92 per index that is a few columns
    assert int(res.rank_h[b]) <= k_opt + 4 + k_opt // 10, (b, int(res.rank_h[b]), k_opt)
    if u.shape[1]:
        assert np.abs(u.T @ u - np.eye(u.shape[1])).max() <= 1e-5
        assert np.abs(v.T @ v - np.eye(v.shape[1])).max() <= 1e-5
    if compare_oracle and u.shape[1]:
        l = int(res.samples_h[b])
        k = min(a.shape)
        if l < k:
            _, so, _, _ = O.rsvd(a, SEED, b, l, 1)
        else:
            _, so, _, _, _ = O.svd(a)
        kk = len(s)
        assert np.abs(s - so[:kk]).max() <= 1e-5 * so[0], (b, np.abs(s - so[:kk]).max() / so[0])


def test_rsvd_uneven_blocks_with_rank_hint(bs):
    """128 blocks of the uneven workload (m, n in {64, 128, 256}, sigma_i = exp(-i/r0))."""
    rb = gen.rsvd_uneven_blocks(batch=128)
    res = _run(bs, rb, rb.extra["rank_hint"])
    full = res.samples_h == np.minimum(rb.m, rb.n)
    fallback = (res.info_h & (1 << 22)) != 0
    assert np.all(res.info_h >= 0)
    assert np.all(res.info_h[~full] & 0xff >= 1) and np.all(res.info_h[full & ~fallback] & 0xff == 0)
    for b in range(rb.batch):
        _check_block(rb, res, b)


def test_rsvd_plain_adaptive_without_hint(bs):
    """No rank guess: 8 samples, then 8 more per round until the posterior estimate passes."""
    rb = gen.rsvd_uneven_blocks(batch=48, sizes=(64, 128))
    res = _run(bs, rb, None, max_rounds=16)
    assert np.any((res.info_h & 0xff) > 1)        # some blocks needed more than one round
    for b in range(rb.batch):
        _check_block(rb, res, b)


def test_rsvd_exact_low_rank_is_recovered(bs):
    rng = np.random.default_rng(5)
    shapes = [(100, 80, 7), (256, 256, 20), (64, 200, 3), (130, 70, 12)]
    ms, ns, mats, sig = [], [], [], []
    for (m, n, r) in shapes:
        uu, _ = np.linalg.qr(rng.standard_normal((m, r)))
        vv, _ = np.linalg.qr(rng.standard_normal((n, r)))
        s_ = np.sort(rng.uniform(0.5, 2.0, r))[::-1]
        mats.append((uu * s_) @ vv.T)
        sig.append(s_)
        ms.append(m)
        ns.append(n)
    rb = gen.RaggedBatch(m=np.array(ms, np.int32), n=np.array(ns, np.int32), offset=None, flat=None)
    sizes = np.array([m * n for m, n in zip(ms, ns)]) + 4
    rb.offset = np.concatenate([[0], np.cumsum(sizes)[:-1]])
    rb.flat = np.zeros(int(sizes.sum()), np.float32)
    for a, o in zip(mats, rb.offset):
        rb.flat[o:o + a.size] = a.T.reshape(-1).astype(np.float32)
    res = _run(bs, rb, [r for (_, _, r) in shapes])
    for b, (m, n, r) in enumerate(shapes):
        u, s, v = _unpack(res, b)
        assert int(res.rank_h[b]) == r, (b, int(res.rank_h[b]))
        assert np.abs(s - sig[b]).max() <= 2e-6 * sig[b][0]
        _check_block(rb, res, b)


def test_rsvd_full_rank_hint_goes_to_jacobi(bs):
    rb = gen.rsvd_uneven_blocks(batch=24, sizes=(64, 128, 256))
    hint = np.minimum(rb.m, rb.n)              # guess = min(m, n): straight to the full SVD
    res = _run(bs, rb, hint)
    assert np.all(res.samples_h == np.minimum(rb.m, rb.n))
    for b in range(rb.batch):
        _check_block(rb, res, b)


def test_rsvd_rank_capped(bs):
    rb = gen.rsvd_uneven_blocks(batch=8, sizes=(128,))
    res = _run(bs, rb, rb.extra["rank_hint"], kmax=np.full(8, 5, np.int32))
    assert np.all(res.rank_h == 5)
    assert np.all(res.info_h & (1 << 21))


def test_rsvd_workspace_errors(bs):
    rb = gen.rsvd_uneven_blocks(batch=6, sizes=(64,))
    flat = torch.from_numpy(rb.flat).cuda()
    A = bs.Batch.packed(flat, rb.offset, rb.m, rb.n)
    need = bs.batched_rsvd_workspace(A, rb.m, rb.n)
    with pytest.raises(bs.BsvdError) as e:
        bs.rsvd(flat, rb.offset, rb.m, rb.n, workspace=torch.empty(64, dtype=torch.uint8, device="cuda"))
    assert e.value.code == bs.ERR_WORKSPACE
    # room for the fixed parts but not for every matrix: the ones past the end are flagged
    short = torch.empty(need - 3 * 4 * 8192, dtype=torch.uint8, device="cuda")
    res = bs.rsvd(flat, rb.offset, rb.m, rb.n, rank_hint=rb.extra["rank_hint"], workspace=short)
    torch.cuda.synchronize()
    info = res.info.cpu().numpy()
    assert info[0] >= 0 and int(res.samples.cpu()[0]) > 0 and info[-1] == bs.INFO_NO_SCRATCH


# ----------------------------------------------------------------------------------------------
# fixed-rank mode (Algorithm 4 as stated), per-matrix tolerances, q power steps, FP64, and the
# adaptive method's decisions against the oracle's adaptive range finder
# ----------------------------------------------------------------------------------------------

def _packed(rb, dtype):
    flat = torch.from_numpy(rb.flat.astype(dtype)).cuda()
    return flat


def _run_mode(bs, rb, dtype, **kw):
    res = bs.rsvd(_packed(rb, dtype), rb.offset, rb.m, rb.n, seed=SEED, **kw)
    torch.cuda.synchronize()
    res.U_h = res.U.cpu().numpy().astype(np.float64)
    res.V_h = res.V.cpu().numpy().astype(np.float64)
    res.S_h = res.S.cpu().numpy().astype(np.float64)
    res.rank_h = res.rank.cpu().numpy()
    res.info_h = res.info.cpu().numpy()
    res.samples_h = res.samples.cpu().numpy()
    return res


def _fp64_blocks(batch, sizes):
    """The uneven generator's blocks rounded to FP64 instead of FP32."""
    return gen.rsvd_uneven_blocks(batch=batch, sizes=sizes, dtype=np.float64)


@pytest.mark.parametrize("dtype,q", [(np.float32, 1), (np.float32, 0), (np.float32, 2), (np.float64, 1)])
def test_rsvd_fixed_rank_matches_the_oracle(bs, dtype, q):
    """rank[b] = k > 0: k + p samples, q power steps, the first k columns (paper Section 7,
    Algorithm 4); sigma and U, V column by column against the oracle's fixed-rank RSVD with the same
    Omega, after sign alignment."""
    sizes = (64, 128, 256) if dtype == np.float32 else (64, 128)
    rb = gen.rsvd_uneven_blocks(batch=24, sizes=sizes) if dtype == np.float32 else _fp64_blocks(16, sizes)
    kk = np.minimum(rb.m, rb.n)
    rng = np.random.default_rng(4)
    k = np.maximum(1, (rb.extra["rank_hint"] * rng.uniform(0.3, 1.1, rb.batch)).astype(np.int32))
    k[0] = kk[0]                         # k + p past min(m, n): the full SVD, k columns kept
    k[1] = max(1, kk[1] - 8)             # k + p = min(m, n) exactly: the full SVD
    lcap = 160 if dtype == np.float32 else 64  # the library's sample caps
    res = _run_mode(bs, rb, dtype, fixed_rank=k, power_iters=q)
    g = 1e-5 if dtype == np.float32 else 1e-12
    c = 256.0 if dtype == np.float32 else 64.0
    for b in range(rb.batch):
        a = rb.a64(b)
        Uo, So, Vo, l = O.rsvd_rank(a, SEED, b, int(k[b]), 8, q, lcap)
        kb = min(int(k[b]), int(kk[b]))
        assert int(res.rank_h[b]) == kb and int(res.samples_h[b]) == l, (b, int(res.rank_h[b]), kb, l)
        assert int(res.info_h[b]) == (0 if l == kk[b] else 1), (b, int(res.info_h[b]))
        u, s, v = _unpack(res, b)
        assert np.abs(s - So).max() <= g * So[0], (b, np.abs(s - So).max() / So[0])
        s_all = O.rsvd(a, SEED, b, l, q)[1] if l < kk[b] else O.svd(a)[1]
        assert vector_errors(u, Uo, So, dtype, c, s_all) <= 1.0, b
        assert vector_errors(v, Vo, So, dtype, c, s_all) <= 1.0, b


def test_rsvd_samples_past_128_columns(bs):
    """256 x 256 blocks with k + p in (128, 160] stay randomized (the FP32 sample cap is 160: the
    small SVD of R_B^T runs in the shared tier with up to 160 columns); k + p = 161 takes the full
    SVD.  Samples, rank and sigma against the oracle's fixed-rank RSVD at the same cap."""
    rb = gen.rsvd_uneven_blocks(batch=6, sizes=(256,))
    k = np.array([121, 125, 140, 150, 152, 153], np.int32)
    res = _run_mode(bs, rb, np.float32, fixed_rank=k, power_iters=1)
    for b in range(rb.batch):
        a = rb.a64(b)
        Uo, So, Vo, l = O.rsvd_rank(a, SEED, b, int(k[b]), 8, 1, 160)
        assert l == (int(k[b]) + 8 if k[b] + 8 <= 160 else 256), (b, l)
        assert int(res.samples_h[b]) == l and int(res.rank_h[b]) == int(k[b]), (b, int(res.samples_h[b]), l)
        u, s, v = _unpack(res, b)
        assert np.abs(s - So).max() <= 1e-5 * So[0], (b, np.abs(s - So).max() / So[0])
        s_all = O.rsvd(a, SEED, b, l, 1)[1] if l < 256 else O.svd(a)[1]
        assert vector_errors(u, Uo, So, np.float32, 256.0, s_all) <= 1.0, b
        assert vector_errors(v, Vo, So, np.float32, 256.0, s_all) <= 1.0, b


def _clear_rank(so, norm2, eps, est2, delta):
    """The truncation rank of the oracle's values, or None when rounding of the singular values
    (delta, absolute) or a factor 2 in the estimate could move it."""
    lo = O.budget_rank(np.maximum(so - delta, 0.0), norm2, eps, est2 / 2)
    hi = O.budget_rank(so + delta, norm2, eps, 2 * est2)
    return lo if lo == hi else None


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_rsvd_adaptive_decisions_match_the_oracle(bs, dtype):
    """Tolerance mode with per-matrix tolerances: rounds, samples and rank equal the oracle's adaptive
    range finder (same Omega and probes) on every block whose round decisions are clear (the
    estimate at least 2x from eps/2 ||A||_F) and whose truncation rank does not move under the
    FP32/FP64 rounding of sigma and a factor 2 in the estimate."""
    sizes = (64, 128, 256) if dtype == np.float32 else (64, 128)
    rb = gen.rsvd_uneven_blocks(batch=48, sizes=sizes) if dtype == np.float32 else _fp64_blocks(24, sizes)
    rng = np.random.default_rng(6)
    tol = rng.choice([1e-3, 1e-4, 1e-5], rb.batch)
    hint = (rb.extra["rank_hint"] // 2).astype(np.int32)
    hint[::5] = 0
    lcap = 160 if dtype == np.float32 else 64  # the library's sample caps
    res = _run_mode(bs, rb, dtype, rank_hint=hint, tol_per=tol, max_rounds=8)
    delta = (2e-6 if dtype == np.float32 else 1e-13)
    compared_rounds = compared_rank = 0
    for b in range(rb.batch):
        a = rb.a64(b)
        r = O.rsvd_adaptive(a, SEED, b, int(hint[b]), float(tol[b]), 8, 1, 8, lcap)
        thr = 0.25 * tol[b] ** 2 * r["norm2"]
        clear = all(e >= 4 * thr or e <= thr / 4 for e in r["est2_round"])
        u, s, v = _unpack(res, b)
        na = math.sqrt(r["norm2"])
        err = np.linalg.norm(a - (u * s) @ v.T) / na
        assert err <= tol[b], (b, err, tol[b])
        if not clear:
            continue
        compared_rounds += 1
        got = (int(res.info_h[b]) & 0xff, int(res.samples_h[b]), bool(res.info_h[b] & (1 << 22)))
        assert got == (r["rounds"], r["samples"], r["fallback"]), (b, got, r["rounds"], r["samples"], r["fallback"])
        kr = _clear_rank(r["S"], r["norm2"], float(tol[b]), r["est2"], delta * r["S"][0])
        if kr is not None:
            compared_rank += 1
            assert int(res.rank_h[b]) == kr == r["rank"], (b, int(res.rank_h[b]), kr, r["rank"])
    assert compared_rounds >= rb.batch // 3 and compared_rank >= rb.batch // 4, (compared_rounds, compared_rank)


def test_rsvd_fp64_tolerance_mode(bs):
    """FP64 randomized SVD to 1e-10: error <= eps on every block, sigma against the oracle's FP64
    fixed-width RSVD with the same samples within 1e-12 normwise."""
    rb = _fp64_blocks(12, (64, 128, 256))
    res = _run_mode(bs, rb, np.float64, rank_hint=rb.extra["rank_hint"], tol=1e-10, max_rounds=8)
    assert np.all(res.info_h >= 0)
    for b in range(rb.batch):
        a = rb.a64(b)
        u, s, v = _unpack(res, b)
        na = np.linalg.norm(a)
        assert np.linalg.norm(a - (u * s) @ v.T) / na <= 1e-10
        if u.shape[1]:
            assert np.abs(u.T @ u - np.eye(u.shape[1])).max() <= 1e-12
            assert np.abs(v.T @ v - np.eye(v.shape[1])).max() <= 1e-12
        l = int(res.samples_h[b])
        so = O.rsvd(a, SEED, b, l, 1)[1] if l < min(a.shape) else O.svd(a)[1]
        assert np.abs(s - so[:len(s)]).max() <= 1e-12 * so[0], b


def test_rsvd_bad_tolerance_flags_the_matrix(bs):
    rb = gen.rsvd_uneven_blocks(batch=4, sizes=(64,))
    tol = np.array([1e-5, -1.0, float("nan"), 1.5])
    res = _run_mode(bs, rb, np.float32, tol_per=tol)
    assert res.info_h[0] >= 0 and list(res.info_h[1:]) == [-1, -1, -1]


@pytest.mark.parametrize("flags", [1, 2, 3])
def test_rsvd_precision_options_match_the_oracle(bs, flags):
    """BSVD_RSVD_SMALL_FP64 (1: the small SVDs in FP64) and BSVD_RSVD_TC_SAMPLING (2: the sample A Omega
    on the tensor cores, TF32 operands, FP32 accumulation, the probes in FP32): fixed-rank sigma against
    the oracle's fixed-rank RSVD at the same l, and in tolerance mode the error gate, Eckart-Young and
    orthogonality on every block, sigma against the oracle at the sample count used.

    The tensor-core sample is A Omega read with 10-bit mantissas: a sample of a slightly different
    Gaussian matrix, so its rank-l approximation A~ differs from the oracle's A^ (exact Omega) by up to
    the two approximations' errors.  By Weyl's inequality |sigma_i(A~) - sigma_i(A^)| <= ||A - A~||_2 +
    ||A - A^||_2: with the TC sample sigma is compared within 1e-5 sigma_1 plus those two errors (each
    measured in FP64), and the TC approximation's error must stay within twice the oracle's (plus
    1e-5 ||A||_2: the same quality of sample)."""
    rb = gen.rsvd_uneven_blocks(batch=32, sizes=(64, 128, 256))
    kk = np.minimum(rb.m, rb.n)
    k = np.maximum(1, (rb.extra["rank_hint"] * 0.7).astype(np.int32))
    res = _run_mode(bs, rb, np.float32, fixed_rank=k, flags=flags)
    assert np.all(res.info_h >= 0)
    for b in range(rb.batch):
        a = rb.a64(b)
        Uo, So, Vo, l = O.rsvd_rank(a, SEED, b, int(k[b]), 8, 1, 128 if flags & 2 else 160)
        assert int(res.samples_h[b]) == l and int(res.rank_h[b]) == min(int(k[b]), int(kk[b]))
        u, s, v = _unpack(res, b)
        tol = 1e-5 * So[0]
        if flags & 2 and l < kk[b]:
            e_o = np.linalg.norm(a - (Uo * So) @ Vo.T, 2)
            e_g = np.linalg.norm(a - (u * s) @ v.T, 2)
            assert e_g <= 2 * e_o + 1e-5 * So[0], (b, e_g, e_o)
            tol += e_o + e_g
        assert np.abs(s - So).max() <= tol, (b, np.abs(s - So).max() / So[0])
    res = _run_mode(bs, rb, np.float32, rank_hint=rb.extra["rank_hint"] // 2, max_rounds=8, flags=flags)
    assert np.all(res.info_h >= 0)
    for b in range(rb.batch):
        _check_block(rb, res, b)
