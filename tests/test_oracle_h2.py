"""Pins for the FP64 reference of the H^2 basis-tree truncation (Section 8.2) -- CPU only.

The truncated basis is checked against what the representation itself fixes: the nested-basis
relation of Section 8.1 expanded explicitly by brute force, closed forms on a two-leaf tree,
exact reproduction when nothing is truncated, orthonormal new bases, a per-node error bound that
follows from the triangle inequality, truncation ranks recomputed from LAPACK singular values of
explicitly formed matrices, and exactly low-rank trees.
"""
import math

import numpy as np
import pytest

from gen.basis_tree import chebyshev_basis_tree
from oracle.h2 import truncate_basis_tree


def expand(leaves, transfers, l, i):
    """Explicit basis of node i at level l from the leaves and the transfers (Section 8.1)."""
    d = len(transfers) - 1
    if l == d:
        return np.asarray(leaves[i], dtype=np.float64)
    return np.vstack([expand(leaves, transfers, l + 1, 2 * i) @ transfers[l + 1][2 * i],
                      expand(leaves, transfers, l + 1, 2 * i + 1) @ transfers[l + 1][2 * i + 1]])


def brute_rank(s, eps):
    """Smallest k with sqrt(sum_{j >= k} s_j^2) <= eps ||s||, by trying every k."""
    s = np.sort(np.asarray(s, dtype=np.float64))[::-1]
    norm = math.sqrt(float((s * s).sum()))
    for k in range(len(s) + 1):
        if math.sqrt(float((s[k:] ** 2).sum())) <= eps * norm:
            return k
    return len(s)


def random_tree(depth, m, k, seed, decay=0.6, leaf_rank=None):
    """Leaves m x k with singular values decay^j (or exact rank ``leaf_rank``); transfers k x k
    with columns scaled by decay^j, so that truncation also happens above the leaves."""
    rng = np.random.default_rng(seed)
    leaves = []
    for _ in range(2 ** depth):
        r = k if leaf_rank is None else leaf_rank
        x, _ = np.linalg.qr(rng.standard_normal((m, min(m, k))))
        y, _ = np.linalg.qr(rng.standard_normal((k, min(m, k))))
        s = decay ** np.arange(min(m, k))
        s[r:] = 0.0
        leaves.append((x * s) @ y.T)
    transfers = [[]] + [[rng.standard_normal((k, k)) * decay ** np.arange(k) / math.sqrt(k) for _ in range(2 ** l)]
                        for l in range(1, depth + 1)]
    return leaves, transfers


def test_generator_nested_relation():
    tree = chebyshev_basis_tree(3, side=24, q=4)
    for l in range(tree.depth + 1):
        for i in range(2 ** l):
            direct = tree.direct(l, i)
            assert np.abs(expand(tree.leaves, tree.transfers, l, i) - direct).max() <= 1e-13 * np.abs(direct).max()


def test_two_leaf_closed_form():
    a, b, c, d, e1, e2 = 3.0, 4.0, -1.0, 2.0, 0.5, -2.0
    leaves = [np.array([[a], [b]]), np.array([[c], [d]])]
    transfers = [[], [np.array([[e1]]), np.array([[e2]])]]
    nl, nt, T, ranks = truncate_basis_tree(leaves, transfers, 1e-12)
    assert ranks == [[1], [1, 1]]
    n1, n2 = math.hypot(a, b), math.hypot(c, d)
    # leaves: U = sigma u, so the new leaf is +-u and T = +-sigma with the same sign
    assert abs(abs(T[1][0][0, 0]) - n1) < 1e-14 and abs(abs(T[1][1][0, 0]) - n2) < 1e-14
    assert np.allclose(nl[0][:, 0] * np.sign(T[1][0][0, 0]), [a / n1, b / n1], atol=1e-15)
    # root: TE = [T1 e1; T2 e2], sigma = sqrt((n1 e1)^2 + (n2 e2)^2), E~ = TE / sigma up to one sign
    sr = math.hypot(n1 * e1, n2 * e2)
    assert abs(abs(T[0][0][0, 0]) - sr) < 1e-14
    assert abs(abs(nt[1][0][0, 0]) - n1 * abs(e1) / sr) < 1e-15
    assert abs(abs(nt[1][1][0, 0]) - n2 * abs(e2) / sr) < 1e-15
    root = expand(nl, nt, 0, 0) @ T[0][0]
    assert np.abs(root - np.array([[a * e1], [b * e1], [c * e2], [d * e2]])).max() < 1e-14


def test_no_truncation_reproduces_every_node():
    tree = chebyshev_basis_tree(3, side=24, q=4)           # 72 points per leaf, rank 16
    nl, nt, T, ranks = truncate_basis_tree(tree.leaves, tree.transfers, 0.0)
    for l in range(tree.depth + 1):
        for i in range(2 ** l):
            u = expand(tree.leaves, tree.transfers, l, i)
            ut = expand(nl, nt, l, i)
            assert ranks[l][i] == 16
            assert np.abs(ut @ T[l][i] - u).max() <= 1e-12 * np.abs(u).max()
            assert np.abs(ut.T @ ut - np.eye(ranks[l][i])).max() <= 1e-13


@pytest.mark.parametrize("eps,decay", [(1e-2, 0.6), (1e-5, 0.3)])
def test_orthonormal_bases_optimal_ranks_and_error_bound(eps, decay):
    depth, m, k = 3, 20, 12
    leaves, transfers = random_tree(depth, m, k, seed=1, decay=decay)
    nl, nt, T, ranks = truncate_basis_tree(leaves, transfers, eps)
    bound = {}
    for l in range(depth, -1, -1):
        for i in range(2 ** l):
            u = expand(leaves, transfers, l, i)
            ut = expand(nl, nt, l, i)
            r = ranks[l][i]
            assert ut.shape[1] == r and T[l][i].shape == (r, k)
            assert np.abs(ut.T @ ut - np.eye(r)).max(initial=0.0) <= 1e-13
            if l == depth:
                s = np.linalg.svd(u, compute_uv=False)
                bound[l, i] = eps * np.linalg.norm(u)
            else:
                # the truncated matrix is TE, whose singular values are those of U_p projected on
                # the children's new bases (the children's bases are orthonormal)
                kids = [expand(nl, nt, l + 1, c) for c in (2 * i, 2 * i + 1)]
                proj = np.vstack([kids[0] @ kids[0].T @ u[:len(kids[0])], kids[1] @ kids[1].T @ u[len(kids[0]):]])
                s = np.linalg.svd(proj, compute_uv=False)
                bc = math.sqrt(sum((bound[l + 1, c] * np.linalg.norm(transfers[l + 1][c], 2)) ** 2
                                   for c in (2 * i, 2 * i + 1)))
                bound[l, i] = bc + eps * (np.linalg.norm(u) + bc)
            assert r == brute_rank(s, eps), (l, i, r, brute_rank(s, eps))
            err = np.linalg.norm(u - ut @ T[l][i])
            assert err <= bound[l, i] * (1 + 1e-9) + 1e-13 * np.linalg.norm(u), (l, i, err, bound[l, i])
    # truncation does happen above the leaves for this tree
    assert min(ranks[0]) < k and min(min(r) for r in ranks[1:depth]) < k


def test_exactly_low_rank_tree():
    depth, m, k, r = 3, 16, 10, 3
    leaves, transfers = random_tree(depth, m, k, seed=7, decay=1.0, leaf_rank=r)
    nl, nt, T, ranks = truncate_basis_tree(leaves, transfers, 1e-10)
    assert ranks[depth] == [r] * 2 ** depth
    for l in range(depth + 1):
        for i in range(2 ** l):
            u = expand(leaves, transfers, l, i)
            s = np.linalg.svd(u, compute_uv=False)
            assert ranks[l][i] == int(np.sum(s > 1e-9 * s[0]))
            assert np.linalg.norm(u - expand(nl, nt, l, i) @ T[l][i]) <= 1e-12 * np.linalg.norm(u)


def test_zero_leaf_gives_rank_zero():
    leaves, transfers = random_tree(2, 8, 6, seed=3)
    leaves[1] = np.zeros_like(leaves[1])
    nl, nt, T, ranks = truncate_basis_tree(leaves, transfers, 1e-8)
    assert ranks[2][1] == 0 and nl[1].shape == (8, 0) and T[2][1].shape == (0, 6)
    assert nt[2][1].shape[0] == 0
    u = expand(leaves, transfers, 0, 0)
    assert np.linalg.norm(u - expand(nl, nt, 0, 0) @ T[0][0]) <= 1e-7 * np.linalg.norm(u)


def test_uneven_chebyshev_leaves_are_truncated_to_their_point_count():
    tree = chebyshev_basis_tree(4, side=28, q=5)           # 784 points: leaves of about 49 > 25, and
    tree2 = chebyshev_basis_tree(4, side=18, q=5)          # 324 points: leaves of about 20 < 25
    for t in (tree, tree2):
        nl, nt, T, ranks = truncate_basis_tree(t.leaves, t.transfers, 1e-7)
        m = [e - s for s, e in t.ranges[t.depth]]
        assert ranks[t.depth] == [min(mi, 25) for mi in m]
