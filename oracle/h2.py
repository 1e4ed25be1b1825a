"""FP64 reference for the truncation phase of H^2-matrix compression (test infrastructure only).

Section 8.2 of Boukaram et al. (2017): a nested row basis -- explicit leaf bases U^d_i and, for
every non-root node c, a transfer matrix E^l_c with U^{l-1}_p = diag(U^l_{2p}, U^l_{2p+1})
[E^l_{2p}; E^l_{2p+1}] (Section 8.1) -- is replaced level by level by a truncated, orthonormal
nested basis (leaves Ũ, transfers Ẽ) together with the projection matrices T = Ũ^T U of every
node.  Steps, in the paper's order and notation:

  1. every leaf i: SVD U^d_i = Q S W^T; keep the leading k̃ singular triplets, k̃ the smallest
     rank whose discarded tail is within eps ||U^d_i||_F; Ũ^d_i = Q̃ and T^d_i = Ũ^d_i^T U^d_i;
  2. level l = d, d-1, ..., 1, every parent p at level l-1 (children c1 = 2p, c2 = 2p + 1):
     TE_p = [T^l_{c1} E^l_{c1}; T^l_{c2} E^l_{c2}]; SVD TE_p = Q S W^T, truncated as in 1;
     Ẽ^l_{c1} and Ẽ^l_{c2} are the first k̃^l_{c1} and the next k̃^l_{c2} rows of Q̃, and
     T^{l-1}_p = S̃ W̃^T.

Every SVD is the oracle's one-sided Jacobi (Algorithm 2) and the truncation rank the oracle's
``trunc_rank``; the products are plain numpy matrix products.  Readings where the paper is
silent: the relative threshold of each node is taken against the Frobenius norm of the matrix
whose SVD is truncated (the leaf basis, or TE); the sweep runs to the root (level 0), whose T is
returned with the rest.  Nothing here is shared with the CUDA library.
"""
from __future__ import annotations

import numpy as np

from . import svd, trunc_rank


def _truncated_svd(a, eps: float):
    """(Q̃, s̃, W̃, k̃) of ``a``: the leading singular triplets kept by the relative threshold."""
    q, s, w, info, _ = svd(a, max_sweeps=60)
    if info < 0 or info >= (1 << 20):
        raise RuntimeError(f"oracle Jacobi did not converge on a {a.shape} node matrix (info {info})")
    k = trunc_rank(s, float(np.sqrt((s * s).sum())), eps) if s.size else 0
    return q[:, :k], s[:k], w[:, :k], k


def truncate_basis_tree(leaves, transfers, eps: float):
    """Truncation phase of Section 8.2.

    ``leaves``: list of the 2^d leaf bases U^d_i (m_i x k_i); ``transfers``: list indexed by level
    (``transfers[0]`` unused), ``transfers[l][c]`` = E^l_c (k^l_c x k^{l-1}_{c // 2}).
    Returns (new_leaves, new_transfers, T, ranks): ``new_leaves[i]`` = Ũ^d_i (m_i x k̃^d_i),
    ``new_transfers[l][c]`` = Ẽ^l_c (k̃^l_c x k̃^{l-1}_{c // 2}), ``T[l][i]`` = T^l_i
    (k̃^l_i x k^l_i) for every level l = 0..d, ``ranks[l][i]`` = k̃^l_i."""
    d = len(transfers) - 1
    if len(leaves) != 2 ** d:
        raise ValueError("a tree of depth d has 2^d leaves")
    T = [None] * (d + 1)
    ranks = [None] * (d + 1)
    new_transfers = [[] for _ in range(d + 1)]
    new_leaves, T[d], ranks[d] = [], [], []
    for u in leaves:                                   # step 1: the leaves
        u = np.asarray(u, dtype=np.float64)
        qt, _, _, k = _truncated_svd(u, eps)
        new_leaves.append(qt)
        T[d].append(qt.T @ u)                          # T^d_i = Ũ^T U
        ranks[d].append(k)
    for l in range(d, 0, -1):                          # step 2: sweep up, one level at a time
        T[l - 1], ranks[l - 1] = [], []
        new_transfers[l] = [None] * (2 ** l)
        for p in range(2 ** (l - 1)):
            c1, c2 = 2 * p, 2 * p + 1
            te = np.vstack([T[l][c1] @ transfers[l][c1], T[l][c2] @ transfers[l][c2]])
            qt, st, wt, k = _truncated_svd(te, eps)
            r1 = ranks[l][c1]
            new_transfers[l][c1] = qt[:r1]
            new_transfers[l][c2] = qt[r1:]
            T[l - 1].append(st[:, None] * wt.T)       # T^{l-1}_p = S̃ W̃^T
            ranks[l - 1].append(k)
    return new_leaves, new_transfers, T, ranks
