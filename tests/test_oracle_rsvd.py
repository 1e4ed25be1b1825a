"""Pins for the oracle's sampling matrix and randomized SVD (Algorithm 4, Section 7) -- CPU only."""
import math
import os

import numpy as np
import pytest

import gen
import oracle as O


def _kat(golden_dir):
    rows = []
    with open(os.path.join(golden_dir, "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            w = [int(x, 16) for x in line.split()]
            rows.append((w[0:4], w[4:6], w[6:10]))
    return rows


def test_philox_known_answers(golden_dir):
    rows = _kat(golden_dir)
    assert len(rows) == 3
    for ctr, key, out in rows:
        assert list(O.philox4x32_10(ctr, key)) == out


def test_gaussian_stream_statistics():
    from scipy import stats
    z = O.omega(12345, 7, 0, 4096, 0, 8).reshape(-1)
    assert abs(z.mean()) < 4.0 / math.sqrt(z.size)
    assert abs(z.var() - 1.0) < 6.0 * math.sqrt(2.0 / z.size)
    assert stats.kstest(z, "norm").pvalue > 1e-3
    # different tag, index or seed -> a different stream
    z2 = O.omega(12345, 8, 0, 64, 0, 1)
    z3 = O.omega(12345, 7, 1, 64, 0, 1)
    z4 = O.omega(12346, 7, 0, 64, 0, 1)
    for other in (z2, z3, z4):
        assert not np.allclose(O.omega(12345, 7, 0, 64, 0, 1), other)


def test_gaussian_box_muller_pairs_share_a_radius():
    # rows 4g, 4g+1 come from words (w0, w1); rows 4g+2, 4g+3 from (w2, w3)
    seed, idx = 99, 3
    w = O.philox4x32_10([5, 2, idx, 0], [seed & 0xFFFFFFFF, seed >> 32])
    col = O.omega(seed, idx, 0, 24, 2, 1)[:, 0]
    for pair, (wa, _) in enumerate([(w[0], w[1]), (w[2], w[3])]):
        za, zb = col[20 + 2 * pair], col[21 + 2 * pair]
        ua = (float(wa) + 0.5) / 2.0 ** 32
        assert abs(za * za + zb * zb + 2.0 * math.log(ua)) < 1e-12


def test_omega_columns_are_prefix_stable():
    a = O.omega(1, 2, 0, 50, 0, 12)
    b = O.omega(1, 2, 0, 50, 8, 4)
    assert np.array_equal(a[:, 8:], b)


@pytest.mark.parametrize("m,n,r,l", [(40, 30, 5, 8), (64, 64, 10, 13), (30, 50, 3, 6)])
def test_rsvd_exact_rank_input_is_recovered(m, n, r, l):
    rng = np.random.default_rng(m + n + r)
    u, _ = np.linalg.qr(rng.standard_normal((m, r)))
    v, _ = np.linalg.qr(rng.standard_normal((n, r)))
    s_true = np.sort(rng.uniform(0.5, 3.0, r))[::-1]
    a = (u * s_true) @ v.T
    U, S, V, info = O.rsvd(a, seed=5, index=0, l=l, q=1)
    assert np.abs(S[:r] - s_true).max() < 1e-13
    assert np.abs(S[r:]).max() < 1e-13
    assert np.linalg.norm(a - (U[:, :r] * S[:r]) @ V[:, :r].T) < 1e-13 * np.linalg.norm(a)
    assert np.abs(U.T @ U - np.eye(l)).max() < 1e-12 or r < l  # trailing vectors span noise


def test_rsvd_full_width_equals_svd():
    b = gen.uniform_batch(9, 1, 24, 20, np.float64, lambda i: np.exp(-np.arange(20) / 3.0))
    a = b.a64(0)
    U, S, V, info = O.rsvd(a, seed=1, index=0, l=20, q=0)
    assert np.abs(S - b.sigma[0]).max() < 1e-14
    assert np.linalg.norm(a - (U * S) @ V.T) < 1e-14 * np.linalg.norm(a)
    assert np.abs(U.T @ U - np.eye(20)).max() < 1e-13
    assert np.abs(V.T @ V - np.eye(20)).max() < 1e-13


def test_rsvd_error_bounded_below_by_eckart_young():
    """No rank-k approximation beats the truncated SVD (Section 1: the unique minimiser)."""
    b = gen.rsvd_uneven_blocks(batch=6)
    for i in range(b.batch):
        a = b.a64(i)
        k_full = min(a.shape)
        s = b.sigma[i]
        for l in (4, 10, min(20, k_full)):
            U, S, V, info = O.rsvd(a, seed=77, index=i, l=l, q=1)
            for k in (1, l // 2, l):
                err = np.linalg.norm(a - (U[:, :k] * S[:k]) @ V[:, :k].T)
                opt = math.sqrt(float(np.sum(s[k:] ** 2)))
                assert err >= opt * (1 - 1e-9) - 1e-14 * np.linalg.norm(a)


def test_power_step_improves_the_basis():
    b = gen.uniform_batch(10, 1, 128, 96, np.float64, lambda i: np.exp(-np.arange(96) / 10.0))
    a = b.a64(0)
    om = O.omega(3, 0, 0, 96, 0, 30)
    errs = []
    for q in (0, 1, 2):
        Q = O.range_basis(a, om, q)
        assert np.abs(Q.T @ Q - np.eye(30)).max() < 1e-13
        errs.append(np.linalg.norm(a - Q @ (Q.T @ a)))
    assert errs[1] < errs[0] and errs[2] < errs[1]
    assert errs[0] >= math.sqrt(np.sum(b.sigma[0][30:] ** 2)) * (1 - 1e-9)


@pytest.mark.parametrize("seed", range(6))
def test_trunc_rank_brute_force(seed):
    rng = np.random.default_rng(seed)
    s = np.sort(np.exp(rng.uniform(-14, 0, 40)))[::-1]
    na = float(np.sqrt(np.sum(s ** 2))) * rng.uniform(1.0, 1.2)
    for eps in (1e-1, 1e-3, 1e-5, 1e-8, 0.0):
        want = next(k for k in range(len(s) + 1) if math.sqrt(float(np.sum(s[k:] ** 2))) <= eps * na)
        assert O.trunc_rank(s, na, eps) == want


# ----------------------------------------------------------------------------------------------
# adaptive range finder (Halko, Martinsson & Tropp 2011, Sec. 4.3-4.4, around Algorithm 4)
# ----------------------------------------------------------------------------------------------

def _spectrum_matrix(m, n, sig, seed):
    """A = U diag(sig) V^T with Haar U, V (numpy QR of Gaussians, sign-fixed)."""
    rng = np.random.default_rng(seed)
    k = len(sig)
    u, r = np.linalg.qr(rng.standard_normal((m, k)))
    u *= np.sign(np.diag(r))
    v, r = np.linalg.qr(rng.standard_normal((n, k)))
    v *= np.sign(np.diag(r))
    return (u * np.asarray(sig)) @ v.T


def test_posterior_estimate_single_entry_closed_form():
    # E = A - U S V^T = c e_i e_j^T  =>  ||E w||^2 = c^2 w_j^2, so est^2 = c^2 mean_p w_p(j)^2 over the
    # 8 probe columns of stream 1 (not stream 0, which is Omega)
    m, n, i, j, c = 12, 9, 4, 6, 3.0
    a = np.zeros((m, n))
    a[i, j] = c
    u = np.zeros((m, 1))
    v = np.zeros((n, 1))
    s = np.zeros(1)
    seed, idx = 77, 5
    w = O.omega(seed, idx, 1, n, 0, 8)
    want = c * c * np.mean(w[j, :] ** 2)
    got = O.post_est2(a, u, s, v, seed, idx)
    assert abs(got - want) <= 1e-14 * want
    assert abs(got - c * c * np.mean(O.omega(seed, idx, 0, n, 0, 8)[j, :] ** 2)) > 1e-6 * want


def test_posterior_estimate_is_unbiased():
    # E[est^2] = ||A - U S V^T||_F^2 for Gaussian probes; averaged over 400 independent probe sets
    # (3200 probes) the relative standard deviation is at most sqrt(2 / 3200) = 0.025
    a = _spectrum_matrix(40, 30, np.exp(-np.arange(30) / 4.0), 3)
    U, S, V, _ = O.rsvd(a, seed=1, index=0, l=6, q=0)
    exact = np.linalg.norm(a - (U * S) @ V.T) ** 2
    ests = [O.post_est2(a, U, S, V, seed, 0) for seed in range(1000, 1400)]
    assert abs(np.mean(ests) - exact) <= 0.1 * exact
    # an exact factorisation has a zero estimate
    u, s, vt = np.linalg.svd(a, full_matrices=False)
    assert O.post_est2(a, u, s, vt.T, 9, 0) <= 1e-26 * np.linalg.norm(a) ** 2


def test_budget_rank_brute_force():
    rng = np.random.default_rng(2)
    for _ in range(200):
        s = np.sort(rng.uniform(0, 1, 30) ** 6)[::-1]
        n2 = float(np.sum(s ** 2)) * rng.uniform(1.0, 1.5)
        eps = 10.0 ** rng.uniform(-3, -0.5)
        est2 = rng.uniform(0, 0.3) * eps * eps * n2
        thr = max(0.0, 0.9025 * eps * eps * n2 - 4.0 * est2)
        want = min(k for k in range(31) if np.sum(s[k:] ** 2) <= thr)
        assert O.budget_rank(s, n2, eps, est2) == want


def test_adaptive_exact_rank_accepted_in_one_round():
    sig = np.r_[np.linspace(2.0, 1.0, 12), np.zeros(48)]
    a = _spectrum_matrix(80, 60, sig, 7)
    r = O.rsvd_adaptive(a, seed=11, index=3, hint=12, eps=1e-5)
    assert (r["rounds"], r["samples"], r["fallback"], r["rank"]) == (1, 20, False, 12)
    assert r["est2"] <= 1e-24 * r["norm2"]
    assert np.abs(r["S"][:12] - sig[:12]).max() <= 1e-13


def test_adaptive_grows_the_sample_until_accepted():
    # 12 unit values, then a gap to 1e-9: 8 samples miss four directions (est ~ 2 / sqrt(12) ||A||),
    # 16 capture all of them (est ~ 1e-9): two rounds, 16 samples, rank 12
    sig = np.r_[np.ones(12), np.full(38, 1e-9)]
    a = _spectrum_matrix(70, 50, sig, 8)
    r = O.rsvd_adaptive(a, seed=12, index=0, hint=0, eps=1e-5, max_rounds=8)
    assert (r["rounds"], r["samples"], r["fallback"], r["rank"]) == (2, 16, False, 12)
    assert r["est2_round"][0] > 0.25 * 1e-10 * r["norm2"] >= r["est2_round"][1]


def test_adaptive_rejects_an_estimate_between_half_eps_and_eps():
    # rank 10 plus a flat tail of relative norm 0.7 eps over 70 values: a rank-l approximation
    # leaves at least 70 - (l - 10) tail values, 0.7 sqrt((80 - l) / 70) eps >= 0.57 eps for
    # l <= 34, so est^2 ~ 0.33-0.43 eps^2 (8 probes of a flat residual spread it by ~6%) stays
    # above (eps/2)^2 in all three rounds and the method ends in the full SVD; an acceptance rule
    # at eps instead of eps/2 would stop in round 1
    eps = 1e-5
    t = 0.7 * eps * np.sqrt(10.0) / np.sqrt(70.0)
    sig = np.r_[np.ones(10), np.full(70, t)]
    a = _spectrum_matrix(90, 80, sig, 9)
    r = O.rsvd_adaptive(a, seed=13, index=1, hint=10, eps=eps, max_rounds=3)
    assert r["rounds"] == 3 and r["fallback"] and r["samples"] == 80
    assert all(e > 0.25 * eps * eps * r["norm2"] for e in r["est2_round"])
    # the full SVD's truncation keeps what the budget needs
    k = r["rank"]
    err = np.linalg.norm(a - (r["U"][:, :k] * r["S"][:k]) @ r["V"][:, :k].T) / np.linalg.norm(a)
    assert err <= 0.95 * eps


def test_adaptive_falls_back_when_the_sample_would_reach_min_mn():
    a = _spectrum_matrix(20, 20, np.ones(20), 10)
    r = O.rsvd_adaptive(a, seed=1, index=0, hint=10, eps=1e-5)   # l = 18, next 26 >= 20
    assert (r["rounds"], r["samples"], r["fallback"], r["rank"]) == (1, 20, True, 20)
    r = O.rsvd_adaptive(a, seed=1, index=0, hint=12, eps=1e-5)   # l = 20 = min(m, n): full at once
    assert (r["rounds"], r["samples"], r["fallback"]) == (0, 20, False)
    c = _spectrum_matrix(26, 26, np.ones(26), 13)
    r = O.rsvd_adaptive(c, seed=1, index=0, hint=10, eps=1e-5)   # l = 18, next 26 = min(m, n)
    assert (r["rounds"], r["samples"], r["fallback"]) == (1, 26, True)
    b = _spectrum_matrix(200, 200, np.exp(-np.arange(200) / 30.0), 11)
    r = O.rsvd_adaptive(b, seed=1, index=0, hint=121, eps=1e-5)  # l = 129 > 128: full at once
    assert (r["rounds"], r["samples"], r["fallback"]) == (0, 200, False)


_RB = {}


@pytest.mark.parametrize("b", range(0, 24, 3))
def test_adaptive_meets_the_tolerance_above_the_optimum(b):
    # generator blocks with half the generator's rank hint: error <= eps and rank >= Eckart-Young's
    if "rb" not in _RB:
        _RB["rb"] = gen.rsvd_uneven_blocks(batch=24, sizes=(64, 128))
    rb = _RB["rb"]
    a = rb.a64(b)
    eps = 1e-5
    r = O.rsvd_adaptive(a, seed=21, index=b, hint=int(rb.extra["rank_hint"][b]) // 2, eps=eps, max_rounds=8)
    k = r["rank"]
    na = np.linalg.norm(a)
    err = np.linalg.norm(a - (r["U"][:, :k] * r["S"][:k]) @ r["V"][:, :k].T) / na
    assert err <= eps
    sv = np.linalg.svd(a, compute_uv=False)
    assert k >= O.trunc_rank(sv, na, eps)
    assert abs(r["norm2"] - na * na) <= 1e-13 * na * na


def test_fixed_rank_is_algorithm_4_truncated():
    a = _spectrum_matrix(60, 50, np.exp(-np.arange(50) / 5.0), 12)
    U, S, V, l = O.rsvd_rank(a, seed=3, index=2, k=10, p=8, q=1)
    assert l == 18 and U.shape == (60, 10) and V.shape == (50, 10) and S.shape == (10,)
    Uf, Sf, Vf, _ = O.rsvd(a, 3, 2, 18, 1)
    assert np.array_equal(S, Sf[:10]) and np.array_equal(U, Uf[:, :10]) and np.array_equal(V, Vf[:, :10])
    sv = np.linalg.svd(a, compute_uv=False)
    assert np.abs(S - sv[:10]).max() <= 1e-6 * sv[0]       # sigma_19 / sigma_1 = e^-3.6: one power step
    U, S, V, l = O.rsvd_rank(a, seed=3, index=2, k=45, p=8, q=1)   # 53 >= 50: the full SVD, 45 kept
    assert l == 50 and np.abs(S - sv[:45]).max() <= 1e-13
    _, s_full, _, _, _ = O.svd(a)
    U, S, V, l = O.rsvd_rank(a, seed=3, index=2, k=42, p=8, q=1)   # 50 = min(m, n): the full SVD itself
    assert l == 50 and np.array_equal(S, s_full[:42])
