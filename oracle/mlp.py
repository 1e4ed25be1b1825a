"""FP64 reference for the learned rank predictor (test infrastructure only).

The network is the one the CUDA library implements: y = w3 . relu(W2 relu(W1 f + b1) + b2) + b3
with loss L = 1/(2B) sum_b (y_b - t_b)^2; parameters packed as W1 (64 x 16, row-major), b1, W2
(64 x 64), b2, w3 (64), b3.  The features are written from their definition with the oracle's own
Philox/Box-Muller Gaussian stream 2.  No part of this module is shared with the CUDA code.
"""
from __future__ import annotations

import math

import numpy as np

F, H = 16, 64
SIZES = [("W1", H * F), ("b1", H), ("W2", H * H), ("b2", H), ("w3", H), ("b3", 1)]
NPARAMS = sum(s for _, s in SIZES)


def unpack(p):
    p = np.asarray(p, dtype=np.float64)
    out, o = {}, 0
    for name, size in SIZES:
        out[name] = p[o:o + size]
        o += size
    out["W1"] = out["W1"].reshape(H, F)
    out["W2"] = out["W2"].reshape(H, H)
    return out


def forward(p, X):
    """Outputs y (B,) and the activations (h1, h2) for features X (B x 16)."""
    q = unpack(p)
    X = np.asarray(X, dtype=np.float64)
    z1 = X @ q["W1"].T + q["b1"]
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ q["W2"].T + q["b2"]
    h2 = np.maximum(z2, 0.0)
    y = h2 @ q["w3"] + q["b3"][0]
    return y, (X, z1, h1, z2, h2)


def loss_and_grad(p, X, t):
    """L = 1/(2B) sum (y - t)^2 and dL/dp by backpropagation (chain rule layer by layer)."""
    q = unpack(p)
    y, (X, z1, h1, z2, h2) = forward(p, X)
    B = len(y)
    r = y - np.asarray(t, dtype=np.float64)
    L = 0.5 * float(r @ r) / B
    dy = r / B
    g_w3 = h2.T @ dy
    g_b3 = np.array([dy.sum()])
    d2 = np.outer(dy, q["w3"]) * (z2 > 0)
    g_W2 = d2.T @ h1
    g_b2 = d2.sum(0)
    d1 = (d2 @ q["W2"]) * (z1 > 0)
    g_W1 = d1.T @ X
    g_b1 = d1.sum(0)
    g = np.concatenate([g_W1.reshape(-1), g_b1, g_W2.reshape(-1), g_b2, g_w3, g_b3])
    return L, g


def init_params(seed: int = 0):
    """He-style initialisation (the same recipe the training module uses; any start point works)."""
    rng = np.random.default_rng(seed)
    W1 = rng.standard_normal((H, F)) * math.sqrt(2.0 / F)
    W2 = rng.standard_normal((H, H)) * math.sqrt(2.0 / H)
    w3 = rng.standard_normal(H) * math.sqrt(1.0 / H)
    return np.concatenate([W1.reshape(-1), np.zeros(H), W2.reshape(-1), np.zeros(H), w3, [1.0]])


def sketch_features(a, seed: int, index: int):
    """The 16 features of one FP64 matrix ``a`` (m x n) from their definitions."""
    from . import omega
    a = np.asarray(a, dtype=np.float64)
    m, n = a.shape
    G = omega(seed, index, 2, n, 0, 8)
    cn = (a * a).sum(0)
    fro2 = cn.sum()
    fro = math.sqrt(fro2)
    r = np.sqrt(cn) / fro
    lr = np.log10(np.maximum(r, 1e-300))
    Y = a @ G
    W = a.T @ Y
    yy = (Y * Y).sum(0)
    ww = (W * W).sum(0)
    y = yy / fro2
    w = ww / (yy * fro2)
    top = max(n // 8, 1)
    etop = np.sort(cn)[::-1][:top].sum()
    rmax = np.sqrt(ww / yy).max()
    l10 = lambda v: math.log10(max(v, 1e-300))
    return np.array([m / 256.0, n / 256.0, l10(fro), l10(r.max()), l10(r.min()), lr.mean(),
                     math.sqrt(max((lr * lr).mean() - lr.mean() ** 2, 0.0)), l10(y.mean()),
                     math.sqrt(((y - y.mean()) ** 2).mean()) / y.mean(), l10(w.mean()), l10(w.max()), l10(w.min()),
                     l10(y.max()), l10(y.min()), l10(fro2 / rmax ** 2), etop / fro2])
