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
