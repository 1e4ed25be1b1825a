"""Pins for the oracle's Householder QR (Algorithm 1, Section 2.1) -- CPU only.

Each pin checks the oracle against something other than itself: LAPACK (numpy.linalg.qr),
closed forms for tiny shapes, and invariants that a dropped term, a wrong sign or a transposed
operand would break.
"""
import numpy as np
import pytest

import gen
import oracle as O


def _signfix(q, r):
    d = np.sign(np.diag(r))
    d[d == 0] = 1.0
    return q * d, r * d[:, None]


@pytest.mark.parametrize("m,n", [(1, 1), (2, 1), (2, 2), (5, 3), (8, 8), (17, 5), (32, 32), (64, 17), (128, 32)])
def test_qr_matches_lapack_after_sign_normalisation(m, n):
    rng = np.random.default_rng(m * 100 + n)
    a = rng.standard_normal((m, n))
    q, r = O.qr(a)
    ql, rl = np.linalg.qr(a)
    q1, r1 = _signfix(q, r)
    q2, r2 = _signfix(ql, rl)
    scale = np.abs(a).max()
    assert np.abs(r1 - r2).max() <= 1e-13 * scale * max(m, 4)
    assert np.abs(q1 - q2).max() <= 1e-12 * max(m, 4)


@pytest.mark.parametrize("m,n", [(32, 32), (128, 32), (40, 7)])
def test_qr_invariants(m, n):
    b = gen.uniform_batch(7, 1, m, n, np.float64, lambda i: np.logspace(0, -6, min(m, n)))
    a = b.a64(0)
    q, r = O.qr(a)
    assert np.abs(q.T @ q - np.eye(n)).max() <= 1e-14 * m
    assert np.linalg.norm(a - q @ r) / np.linalg.norm(a) <= 1e-14 * m
    assert np.all(np.tril(r, -1) == 0.0)          # exact zeros below the diagonal


def test_qr_1x1_and_2x1_closed_forms():
    # house of a 1-vector flips its sign: Q = -1, R = -a
    q, r = O.qr(np.array([[3.5]]))
    assert q[0, 0] == -1.0 and r[0, 0] == -3.5
    q, r = O.qr(np.array([[-2.0]]))
    assert q[0, 0] == -1.0 and r[0, 0] == 2.0
    # 2 x 1: R = -sign(a) sqrt(a^2 + b^2), Q = -sign(a) [a, b] / sqrt(a^2 + b^2)
    a, b = 3.0, 4.0
    q, r = O.qr(np.array([[a], [b]]))
    assert abs(r[0, 0] + 5.0) < 1e-15
    assert np.allclose(q[:, 0], [-0.6, -0.8], atol=1e-15)
    q, r = O.qr(np.array([[-a], [b]]))
    assert abs(r[0, 0] - 5.0) < 1e-15
    assert np.allclose(q[:, 0], [-0.6, 0.8], atol=1e-15)


def test_qr_rank_one():
    rng = np.random.default_rng(3)
    x = rng.standard_normal(9)
    y = rng.standard_normal(4)
    a = np.outer(x, y)
    q, r = O.qr(a)
    s = -np.sign(x[0])
    assert np.allclose(r[0], s * np.linalg.norm(x) * y, atol=1e-13)
    assert np.allclose(q[:, 0], s * x / np.linalg.norm(x), atol=1e-14)
    assert np.abs(r[1:]).max() < 1e-13


def test_qr_orthogonal_columns_gives_diagonal_r():
    rng = np.random.default_rng(5)
    u, _ = np.linalg.qr(rng.standard_normal((12, 6)))
    d = np.array([5.0, 4.0, 3.0, 2.0, 1.0, 0.5])
    a = u * d
    q, r = O.qr(a)
    assert np.allclose(np.abs(np.diag(r)), d, atol=1e-13)
    assert np.abs(np.triu(r, 1)).max() < 1e-13


def test_qr_zero_column_gives_identity_reflector():
    a = np.zeros((5, 3))
    a[:, 1] = [1.0, 2.0, 0.0, 0.0, 2.0]
    q, r = O.qr(a)
    assert np.all(r[:, 0] == 0.0)
    assert np.abs(q @ r - a).max() < 1e-14
    assert np.abs(q.T @ q - np.eye(3)).max() < 1e-14


def test_house_reflects_onto_e1():
    rng = np.random.default_rng(11)
    for x in [rng.standard_normal(7), np.array([0.0, 1.0, -2.0]), np.array([-3.0])]:
        v = O.house(x)
        hx = x - 2.0 * v * (v @ x)
        sgn = 1.0 if x[0] >= 0 else -1.0
        assert abs(hx[0] + sgn * np.linalg.norm(x)) < 1e-14
        assert np.abs(hx[1:]).max(initial=0.0) < 1e-14
        assert abs(np.linalg.norm(v) - 1.0) < 1e-15
    assert np.all(O.house(np.zeros(4)) == 0.0)


def test_qr_batch_equals_single_calls():
    mats = [np.random.default_rng(i).standard_normal((m, n)) for i, (m, n) in enumerate([(4, 4), (9, 2), (6, 6), (3, 1)])]
    qs, rs, info = O.qr_batch(mats, nthreads=3)
    assert np.all(info == 0)
    for a, q, r in zip(mats, qs, rs):
        q1, r1 = O.qr(a)
        assert np.array_equal(q, q1) and np.array_equal(r, r1)
