"""Nested row bases of H^2-matrices built by Chebyshev interpolation (input to the truncation phase).

This module only *makes inputs*; it holds none of the truncation's arithmetic.  The paper's
covariance matrices (Section 8.3) are built by clustering points of a randomly perturbed regular
grid of the unit square with a k-d tree (mean split) and interpolating the kernel on a q x q
Chebyshev grid in every cluster box; their row basis is what the truncation phase compresses.
This is that basis, built from its textbook definition (Boerm, Loehndorf & Melenk 2005):

  * leaf i of the tree (its points x_p, its box B_i): U_i(p, a q + b) = L^{B_i}_a(x_p) L^{B_i}_b(y_p),
    with L^{B}_a the 1D Lagrange polynomials on the q Chebyshev points of the first kind of B's
    side along x (respectively y);
  * node c with parent p: the transfer matrix E_c(a q + b, a' q + b') = L^{B_p}_{a'}(xi^c_a)
    L^{B_p}_{b'}(eta^c_b), the parent's Lagrange polynomials at the child's interpolation points.

Interpolation of a polynomial of degree < q is exact, so U_p = diag(U_{c1}, U_{c2}) [E_{c1}; E_{c2}]
holds to rounding: the nested-basis relation of Section 8.1.  ``direct(l, i)`` evaluates the node's
own Lagrange basis at its points, independently of the transfers, so that a test can check it.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

from . import TAG_MISC, uniforms

WORKLOAD_BASIS_TREE = 5


def cheb_points(lo: float, hi: float, q: int) -> np.ndarray:
    """The q Chebyshev points of the first kind on [lo, hi]."""
    j = np.arange(q, dtype=np.float64)
    return 0.5 * (lo + hi) + 0.5 * (hi - lo) * np.cos((2.0 * j + 1.0) * math.pi / (2.0 * q))


def lagrange(nodes: np.ndarray, x: np.ndarray) -> np.ndarray:
    """L[p, j] = prod_{i != j} (x_p - nodes_i) / (nodes_j - nodes_i)."""
    x = np.asarray(x, dtype=np.float64)
    q = len(nodes)
    out = np.ones((len(x), q))
    for j in range(q):
        for i in range(q):
            if i != j:
                out[:, j] *= (x - nodes[i]) / (nodes[j] - nodes[i])
    return out


def tensor_basis(lo, hi, q: int, pts: np.ndarray) -> np.ndarray:
    """Rows: points; column a q + b: L_a(x) L_b(y) on the box [lo, hi]."""
    lx = lagrange(cheb_points(lo[0], hi[0], q), pts[:, 0])
    ly = lagrange(cheb_points(lo[1], hi[1], q), pts[:, 1])
    return (lx[:, :, None] * ly[:, None, :]).reshape(len(pts), q * q)


def tensor_points(lo, hi, q: int) -> np.ndarray:
    """The q x q interpolation points of a box, point a q + b = (x_a, y_b)."""
    cx, cy = cheb_points(lo[0], hi[0], q), cheb_points(lo[1], hi[1], q)
    return np.stack([np.repeat(cx, q), np.tile(cy, q)], axis=1)


@dataclass
class BasisTree:
    """Row basis over a binary cluster tree of uniform depth ``depth`` (root = level 0).

    Node i of level l owns points ``ranges[l][i]`` (tree order) and box ``boxes[l][i]``; its
    parent is node i // 2 of level l - 1.  ``leaves[i]`` is U^depth_i (m_i x q^2);
    ``transfers[l][i]`` is E^l_i (q^2 x q^2) for l >= 1 (``transfers[0]`` is empty)."""
    depth: int
    q: int
    points: np.ndarray
    ranges: list
    boxes: list
    leaves: list
    transfers: list

    @property
    def k(self) -> int:
        return self.q * self.q

    def direct(self, l: int, i: int) -> np.ndarray:
        """The node's own interpolation basis at its points (not through transfer matrices)."""
        s, e = self.ranges[l][i]
        lo, hi = self.boxes[l][i]
        return tensor_basis(lo, hi, self.q, self.points[s:e])


def perturbed_grid(side: int, seed_index: int = 0, jitter: float = 0.45) -> np.ndarray:
    """side^2 points: cell centres of a regular side x side grid of the unit square, each moved
    by up to ``jitter`` cells along each axis (uniformly)."""
    u = uniforms(WORKLOAD_BASIS_TREE, seed_index, TAG_MISC, 2 * side * side).reshape(side * side, 2)
    i, j = np.meshgrid(np.arange(side), np.arange(side), indexing="ij")
    base = np.stack([i.reshape(-1), j.reshape(-1)], axis=1).astype(np.float64) + 0.5
    return (base + jitter * (2.0 * u - 1.0)) / side


def chebyshev_basis_tree(depth: int, side: int | None = None, q: int = 8, seed_index: int = 0) -> BasisTree:
    """Cluster ``side^2`` perturbed-grid points (default: 64 per leaf on average) with a k-d tree
    of uniform depth, splitting each box at the mean coordinate of its points along the box's
    longer side, and build the Chebyshev-interpolation row basis of rank q^2 on it."""
    if side is None:
        side = int(round(math.sqrt(64 * 2 ** depth)))
    pts = perturbed_grid(side, seed_index)
    perm = np.arange(len(pts))
    ranges = [[(0, len(pts))]]
    boxes = [[(np.zeros(2), np.ones(2))]]
    for l in range(depth):
        nr, nb = [], []
        for (s, e), (lo, hi) in zip(ranges[l], boxes[l]):
            d = int(np.argmax(hi - lo))
            p = pts[perm[s:e]]
            cut = float(p[:, d].mean()) if e > s else 0.5 * (lo[d] + hi[d])
            left = p[:, d] < cut
            order = np.concatenate([np.nonzero(left)[0], np.nonzero(~left)[0]])
            perm[s:e] = perm[s:e][order]
            mid = s + int(left.sum())
            hi0, lo1 = hi.copy(), lo.copy()
            hi0[d] = lo1[d] = cut
            nr += [(s, mid), (mid, e)]
            nb += [(lo, hi0), (lo1, hi)]
        ranges.append(nr)
        boxes.append(nb)
    pts = pts[perm]
    tree = BasisTree(depth=depth, q=q, points=pts, ranges=ranges, boxes=boxes, leaves=[], transfers=[[]])
    tree.leaves = [tree.direct(depth, i) for i in range(2 ** depth)]
    for l in range(1, depth + 1):
        row = []
        for i in range(2 ** l):
            lo_c, hi_c = boxes[l][i]
            lo_p, hi_p = boxes[l - 1][i // 2]
            row.append(tensor_basis(lo_p, hi_p, q, tensor_points(lo_c, hi_c, q)))
        tree.transfers.append(row)
    return tree
