"""GPU parity: truncation of an H^2 nested row basis (Section 8.2) against the FP64 oracle.

The GPU runs the whole tree through the C ABI (bsvd_h2_truncate: batched Jacobi SVDs level by
level); the oracle (``oracle/h2.py``) runs the paper's steps node by node in FP64.  Singular vectors
are unique only up to sign, so every node is compared through sign-free quantities built on the
host in FP64 from the outputs:
  * the truncation rank, wherever the node's singular values put the threshold clearly between
    two ranks (a factor 1.1 either way in the tail);
  * the node's approximation of its original expanded basis, U~_exp T (leaves: U~ T; inner nodes:
    U~_exp = diag(U~_exp(c1), U~_exp(c2)) [E~_c1; E~_c2]), against the oracle's, within 1e-5 (FP32)
    or 1e-11 (FP64) of ||U_exp||_F per level of the tree above the leaves (each level adds one
    truncated SVD's rounding);
  * the orthonormality of every expanded new basis within the same bound.
"""
import math

import numpy as np
import pytest

from gen.basis_tree import chebyshev_basis_tree
from oracle.h2 import truncate_basis_tree

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bs():
    import paper_1707_05141_gb300 as bs
    bs.build()
    assert torch.cuda.is_available()
    return bs


def expand(leaves, transfers, l, i, d):
    if l == d:
        return np.asarray(leaves[i], dtype=np.float64)
    return np.vstack([expand(leaves, transfers, l + 1, 2 * i, d) @ transfers[l + 1][2 * i],
                      expand(leaves, transfers, l + 1, 2 * i + 1, d) @ transfers[l + 1][2 * i + 1]])


def random_tree(depth, m, k, seed, decay=0.6):
    rng = np.random.default_rng(seed)
    leaves = []
    for i in range(2 ** depth):
        mi = m - (i % 5) * 3                         # uneven leaves
        x, _ = np.linalg.qr(rng.standard_normal((mi, min(mi, k))))
        y, _ = np.linalg.qr(rng.standard_normal((k, min(mi, k))))
        leaves.append((x * decay ** np.arange(min(mi, k))) @ y.T)
    transfers = [[]] + [[rng.standard_normal((k, k)) * decay ** np.arange(k) / math.sqrt(k) for _ in range(2 ** l)]
                        for l in range(1, depth + 1)]
    return leaves, transfers


def gpu_tree(res):
    """Host views (FP64) of the GPU's new leaves, transfers, T and ranks, in the oracle's layout."""
    d, k = res.depth, res.k
    rank = res.rank.cpu().numpy()
    flat = res.new_leaf.cpu().numpy().astype(np.float64)
    Tn = res.T.cpu().numpy().astype(np.float64)
    En = res.new_transfer.cpu().numpy().astype(np.float64)
    g = lambda l, i: 2 ** l - 1 + i
    leaves = []
    for i in range(2 ** d):
        m, o, r = int(res.m[i]), int(res.offsets[i]), int(rank[g(d, i)])
        leaves.append(flat[o:o + m * k].reshape(k, m).T[:, :r])
    transfers = [[]]
    for l in range(1, d + 1):
        row = []
        for i in range(2 ** l):
            r, rp = int(rank[g(l, i)]), int(rank[g(l - 1, i // 2)])
            row.append(En[g(l, i)].T[:r, :rp])
        transfers.append(row)
    T = [[Tn[g(l, i)].T[:int(rank[g(l, i)]), :] for i in range(2 ** l)] for l in range(d + 1)]
    ranks = [[int(rank[g(l, i)]) for i in range(2 ** l)] for l in range(d + 1)]
    return leaves, transfers, T, ranks


def _clear_rank(mat, eps):
    """The node's rank when the threshold sits clearly between two ranks (else None)."""
    s = np.linalg.svd(mat, compute_uv=False)
    tot = float((s * s).sum())
    tails = np.concatenate([np.cumsum((s * s)[::-1])[::-1], [0.0]])
    thr = eps * eps * tot
    r = int(np.argmax(tails <= thr))
    ok = (r == 0 or tails[r - 1] > 1.1 * thr) and tails[r] < thr / 1.1
    return r if ok else None


def check(bs, leaves, transfers, k, eps, dtype):
    d = len(transfers) - 1
    dt = np.float32 if dtype == np.float32 else np.float64
    lv = [np.asarray(u).astype(dt).astype(np.float64) for u in leaves]
    tr = [[]] + [[np.asarray(e).astype(dt).astype(np.float64) for e in row] for row in transfers[1:]]
    res = bs.h2_truncate(lv, tr, k, eps, dtype=dt)
    torch.cuda.synchronize()
    info = res.info.cpu().numpy()
    assert np.all((info >= 0) & (info < (1 << 20))), info
    gl, gt, gT, gr = gpu_tree(res)
    ol, ot, oT, orr = truncate_basis_tree(lv, tr, eps)
    g = 1e-5 if dt == np.float32 else 1e-11
    compared = 0
    # matrices each node truncates, from the oracle's (FP64) projections, for the rank margins
    for l in range(d, -1, -1):
        for i in range(2 ** l):
            if l == d:
                mat = lv[i]
            else:
                mat = np.vstack([oT[l + 1][2 * i] @ tr[l + 1][2 * i], oT[l + 1][2 * i + 1] @ tr[l + 1][2 * i + 1]])
            r = _clear_rank(mat, eps)
            if r is not None and r == orr[l][i]:
                compared += 1
                assert gr[l][i] == r, (l, i, gr[l][i], r)
            U = expand(lv, tr, l, i, d)
            nU_g = expand(gl, gt, l, i, d)
            nU_o = expand(ol, ot, l, i, d)
            bound = g * (d - l + 1) * max(np.linalg.norm(U), 1e-300)
            if gr[l][i] == orr[l][i]:
                assert np.abs(nU_g @ gT[l][i] - nU_o @ oT[l][i]).max() <= bound, (l, i)
            if nU_g.shape[1]:
                assert np.abs(nU_g.T @ nU_g - np.eye(nU_g.shape[1])).max() <= g * (d - l + 1), (l, i)
    return compared


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_h2_random_tree(bs, dtype):
    leaves, transfers = random_tree(4, 48, 24, seed=3)
    eps = 1e-4 if dtype == np.float32 else 1e-9
    n = check(bs, leaves, transfers, 24, eps, dtype)
    assert n >= 10, n


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_h2_chebyshev_tree(bs, dtype):
    """The paper's construction (Section 8.3): a k-d tree (mean split) over a perturbed grid of the
    unit square, Chebyshev-interpolation bases of rank q^2 = 64; uneven leaves."""
    tree = chebyshev_basis_tree(5, q=8)
    eps = 1e-5 if dtype == np.float32 else 1e-10
    n = check(bs, tree.leaves, tree.transfers, tree.k, eps, dtype)
    assert n >= 10, n
