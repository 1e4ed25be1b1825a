"""Pins for the oracle's one-sided Jacobi SVD (Algorithm 2, Section 2.2) -- CPU only.

Closed forms (2 x 2 singular values, one rotation zeroing the pair's inner product), special
cases (diagonal input needs no rotation, orthogonal columns, rank one, zero matrix), matrices
built with known singular values, LAPACK's SVD, and the invariants
||U^T U - I||, ||V^T V - I||, ||A - U S V^T|| / ||A||.
"""
import math

import numpy as np
import pytest

import gen
import oracle as O

U64 = 2.0 ** -53


def _closed_form_2x2(a, b, c, d):
    p = math.hypot(a + d, b - c)
    q = math.hypot(a - d, b + c)
    return (p + q) / 2.0, abs(p - q) / 2.0


@pytest.mark.parametrize("seed", range(20))
def test_2x2_closed_form(seed):
    rng = np.random.default_rng(seed)
    a, b, c, d = rng.standard_normal(4) * 10.0 ** rng.uniform(-3, 3)
    A = np.array([[a, b], [c, d]])
    u, s, v, info, _ = O.svd(A)
    s1, s2 = _closed_form_2x2(a, b, c, d)
    assert abs(s[0] - s1) <= 8 * U64 * s1
    assert abs(s[1] - s2) <= 8 * U64 * s1
    assert info >= 1


@pytest.mark.parametrize("seed", range(10))
def test_one_rotation_zeroes_inner_product(seed):
    rng = np.random.default_rng(100 + seed)
    x, y = rng.standard_normal((2, 13))
    y += 0.7 * x
    al, be, ga = x @ x, y @ y, x @ y
    rot, c, s = O.rot(al, be, ga, 1e-15)
    assert rot
    assert abs(c * c + s * s - 1.0) < 4 * U64
    xn = c * x - s * y
    yn = s * x + c * y
    assert abs(xn @ yn) <= 32 * U64 * math.sqrt(al * be)
    # |t| <= 1: the inner rotation
    assert abs(s) <= abs(c) * (1 + 4 * U64)


def test_rot_skips_small_and_zero_columns():
    assert O.rot(1.0, 1.0, 1e-20, 1e-16)[0] is False
    assert O.rot(0.0, 1.0, 0.0, 1e-16)[0] is False
    assert O.rot(1.0, 0.0, 0.0, 1e-16)[0] is False
    # alpha == beta -> zeta = 0 -> t = 1 -> 45 degrees
    rot, c, s = O.rot(2.0, 2.0, 1.0, 1e-16)
    assert rot and abs(c - math.sqrt(0.5)) < 4e-16 and abs(s - math.sqrt(0.5)) < 4e-16


def test_diagonal_needs_no_rotation():
    d = np.array([0.3, -5.0, 2.0, 0.0, 1.0, -0.3])
    u, s, v, info, rots = O.svd(np.diag(d))
    assert rots == 0 and info == 1
    assert np.array_equal(s, np.sort(np.abs(d))[::-1])
    # ties (0.3 and -0.3) keep column order: column 0 first
    assert np.array_equal(np.argsort(-np.abs(d), kind="stable"), np.abs(v).argmax(axis=0))


def test_orthogonal_columns_need_no_rotation():
    rng = np.random.default_rng(2)
    q, _ = np.linalg.qr(rng.standard_normal((20, 8)))
    d = np.array([1.0, 3.0, 2.0, 0.5, 7.0, 0.1, 4.0, 6.0])
    u, s, v, info, rots = O.svd(q * d)
    assert rots == 0
    assert np.allclose(s, np.sort(d)[::-1], rtol=1e-14)


def test_rank_one_and_zero():
    rng = np.random.default_rng(8)
    x, y = rng.standard_normal(10), rng.standard_normal(6)
    u, s, v, info, _ = O.svd(np.outer(x, y))
    assert abs(s[0] - np.linalg.norm(x) * np.linalg.norm(y)) < 1e-13 * s[0]
    assert np.abs(s[1:]).max() < 1e-13 * s[0]
    u, s, v, info, rots = O.svd(np.zeros((5, 4)))
    assert np.all(s == 0.0) and np.all(u == 0.0) and rots == 0


@pytest.mark.parametrize("m,n", [(3, 3), (8, 5), (5, 8), (32, 32), (33, 17), (64, 64), (17, 31)])
def test_against_lapack_and_invariants(m, n):
    rng = np.random.default_rng(m * 1000 + n)
    a = rng.standard_normal((m, n))
    u, s, v, info, _ = O.svd(a)
    k = min(m, n)
    assert info < O.NOT_CONVERGED
    sl = np.linalg.svd(a, compute_uv=False)
    assert np.abs(s - sl).max() <= 1e-14 * sl[0] * max(m, n)
    assert np.all(np.diff(s) <= 0)
    assert np.abs(u.T @ u - np.eye(k)).max() <= 1e-13
    assert np.abs(v.T @ v - np.eye(k)).max() <= 1e-13
    assert np.linalg.norm(a - (u * s) @ v.T) / np.linalg.norm(a) <= 1e-14 * max(m, n)


def test_known_sigma_workload0_matrices():
    """The 32 x 32 FP64 workload with sigma_i = 10^(-8i/31): normwise sigma error ~ u64."""
    b = gen.fp64_32_graded(batch=8)
    for i in range(b.batch):
        a = b.a64(i)
        u, s, v, info, rots = O.svd(a)
        assert info < O.NOT_CONVERGED
        assert np.abs(s - b.sigma[i]).max() / b.sigma[i][0] < 1e-14
        assert np.abs(u.T @ u - np.eye(32)).max() < 1e-13
        assert np.abs(v.T @ v - np.eye(32)).max() < 1e-13
        assert np.linalg.norm(a - (u * s) @ v.T) / np.linalg.norm(a) < 1e-14


def test_singular_vectors_match_lapack_up_to_sign():
    b = gen.svd64_exp8(batch=2)
    a = b.a64(1)
    u, s, v, info, _ = O.svd(a)
    ul, sl, vlt = np.linalg.svd(a)
    for j in range(64):   # distinct, well separated sigma: vectors unique up to sign
        sg = np.sign(u[:, j] @ ul[:, j])
        assert np.abs(u[:, j] - sg * ul[:, j]).max() < 1e-9
        assert np.abs(v[:, j] - sg * vlt[j]).max() < 1e-9


def test_max_sweeps_cap_reports_not_converged():
    rng = np.random.default_rng(1)
    u, s, v, info, rots = O.svd(rng.standard_normal((16, 16)), max_sweeps=1)
    assert info == O.NOT_CONVERGED + 1
    assert rots == 16 * 15 // 2 or rots > 0


def test_svd_batch_matches_single_calls():
    mats = [np.random.default_rng(i).standard_normal(sh) for i, sh in enumerate([(6, 6), (4, 9), (12, 3)])]
    Us, Ss, Vs, info, rots = O.svd_batch(mats, nthreads=2)
    for a, u, s, v, inf in zip(mats, Us, Ss, Vs, info):
        u1, s1, v1, inf1, _ = O.svd(a)
        assert np.array_equal(s, s1) and np.array_equal(u, u1) and np.array_equal(v, v1) and inf == inf1
