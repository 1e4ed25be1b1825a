"""The GPU parity helpers accept correct results and reject wrong ones (CPU only).

The GPU tests judge the CUDA path only through ``tests/parity.py``; these cases feed it LAPACK
factorisations, either as they are (sign choices differing from the oracle's) or with one
planted error each, and check the verdicts.
"""
import numpy as np

import parity as P


def _graded(m, n, seed=0, kappa=1e4):
    rng = np.random.default_rng(seed)
    k = min(m, n)
    u, _ = np.linalg.qr(rng.standard_normal((m, k)))
    v, _ = np.linalg.qr(rng.standard_normal((n, k)))
    s = np.logspace(0, -np.log10(kappa), k)
    return (u * s) @ v.T, s


def test_svd_errors_accept_lapack_and_reject_planted_errors():
    a, s_true = _graded(30, 20)
    u, s, vt = np.linalg.svd(a, full_matrices=False)
    v = vt.T
    ok = P.svd_errors(a, u, s, v, s_true)
    assert max(ok.values()) < 1e-13, ok
    # signs of a (u_j, v_j) pair are free
    u2, v2 = u.copy(), v.copy()
    u2[:, 3] *= -1
    v2[:, 3] *= -1
    assert max(P.svd_errors(a, u2, s, v2, s_true).values()) < 1e-13
    # one sign flipped on U alone breaks the residual
    u3 = u.copy()
    u3[:, 0] *= -1
    assert P.svd_errors(a, u3, s, v, s_true)["resid"] > 1e-5
    # unsorted singular values (two swapped) fail the sigma gate
    s4 = s.copy()
    s4[[0, 1]] = s4[[1, 0]]
    assert P.svd_errors(a, u, s4, v, s_true)["sigma"] > 1e-5
    # a singular value off by 2e-5 of s_1 fails the FP32 gate, by 1e-6 passes it
    s5 = s.copy()
    s5[5] += 2e-5 * s[0]
    assert P.svd_errors(a, u, s5, v, s_true)["sigma"] > P.gate(np.float32)
    s6 = s.copy()
    s6[5] += 1e-6 * s[0]
    assert P.svd_errors(a, u, s6, v, s_true)["sigma"] <= P.gate(np.float32)
    # a non-orthogonal V (two columns mixed) fails the orthogonality check
    v7 = v.copy()
    v7[:, 2] = (v[:, 2] + 1e-4 * v[:, 3]) / np.linalg.norm(v[:, 2] + 1e-4 * v[:, 3])
    assert P.svd_errors(a, u, s, v7, s_true)["orth_v"] > 5e-5


def test_svd_errors_exclude_zero_sigma_columns_from_u():
    a = np.zeros((6, 3))
    a[:, 0] = np.arange(1.0, 7.0)
    u = np.zeros((6, 3))
    u[:, 0] = a[:, 0] / np.linalg.norm(a[:, 0])
    s = np.array([np.linalg.norm(a[:, 0]), 0.0, 0.0])
    v = np.eye(3)
    e = P.svd_errors(a, u, s, v, s)
    assert e["orth_u"] < 1e-15 and e["resid"] < 1e-15 and e["sigma"] == 0.0


def test_vector_errors_sign_free_gap_scaled():
    a, s_true = _graded(25, 12, seed=4, kappa=1e3)
    u, s, _ = np.linalg.svd(a, full_matrices=False)
    flipped = u * np.where(np.arange(12) % 2, -1.0, 1.0)
    assert P.vector_errors(flipped, u, s_true, np.float64) <= 1.0
    # a column moved by 1e-6 is far outside the FP64 allowance, inside the FP32 one
    bad = u.copy()
    bad[:, 4] += 1e-6
    assert P.vector_errors(bad, u, s_true, np.float64) > 1.0
    assert P.vector_errors(bad, u, s_true, np.float32) <= 1.0
    # two swapped columns fail
    sw = u.copy()
    sw[:, [2, 3]] = sw[:, [3, 2]]
    assert P.vector_errors(sw, u, s_true, np.float32) > 1.0
    # a repeated singular value leaves its columns unchecked (only their span is unique)
    s_rep = s_true.copy()
    s_rep[7] = s_rep[6]
    mix = u.copy()
    c, t = np.cos(0.3), np.sin(0.3)
    mix[:, 6], mix[:, 7] = c * u[:, 6] - t * u[:, 7], t * u[:, 6] + c * u[:, 7]
    assert P.vector_errors(mix, u, s_rep, np.float64) <= 1.0


def test_qr_errors_accept_sign_choices_and_reject_planted_errors():
    rng = np.random.default_rng(8)
    a = rng.standard_normal((20, 8))
    q, r = np.linalg.qr(a)
    d = np.where(np.arange(8) % 3 == 0, -1.0, 1.0)     # another valid sign choice
    e = P.qr_errors(a, q * d, r * d[:, None], q, r, np.float64)
    assert e["q"] <= 1.0 and e["r"] <= 1.0 and e["tril_zero"] and e["orth_q"] < 1e-14 and e["resid"] < 1e-14
    r2 = r.copy()
    r2[5, 2] = 1e-300                                   # any non-zero below the diagonal
    assert not P.qr_errors(a, q, r2, q, r, np.float64)["tril_zero"]
    q3 = q.copy()
    q3[:, [1, 2]] = q3[:, [2, 1]]
    e3 = P.qr_errors(a, q3, r, q, r, np.float64)
    assert e3["q"] > 1.0 and e3["resid"] > 1e-3
    r4 = r.copy()
    r4[0, 7] *= 1.0 + 1e-9
    assert P.qr_errors(a, q, r4, q, r, np.float64)["r"] > 1.0
