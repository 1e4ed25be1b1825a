"""Pins for the FP64 reference of the rank predictor (CPU only): backpropagation against central
finite differences, a hand-computed tiny case, and the features against direct definitions."""
import math

import numpy as np

import gen
from oracle import mlp as OM


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(0)
    p = OM.init_params(1) + 0.05 * rng.standard_normal(OM.NPARAMS)
    X = rng.standard_normal((7, 16))
    t = rng.standard_normal(7)
    L, g = OM.loss_and_grad(p, X, t)
    idx = np.concatenate([np.arange(0, OM.NPARAMS, 53), [OM.NPARAMS - 1]])
    for i in idx:
        e = np.zeros(OM.NPARAMS)
        e[i] = 1e-6
        fd = (OM.loss_and_grad(p + e, X, t)[0] - OM.loss_and_grad(p - e, X, t)[0]) / 2e-6
        assert abs(fd - g[i]) <= 1e-7 + 1e-6 * abs(g[i]), (i, fd, g[i])


def test_single_active_path_by_hand():
    # only W1[0,0], W2[0,0], w3[0], b3 non-zero: y = w3 relu(W2 relu(W1 x)) + b3
    p = np.zeros(OM.NPARAMS)
    q = OM.unpack(p)
    p[0] = 2.0                       # W1[0, 0]
    p[64 * 16 + 64] = 3.0            # W2[0, 0]
    p[64 * 16 + 64 + 64 * 64 + 64] = 0.5   # w3[0]
    p[-1] = 1.0                      # b3
    X = np.zeros((2, 16))
    X[0, 0] = 1.0
    X[1, 0] = -1.0                   # ReLU blocks the second sample
    y, _ = OM.forward(p, X)
    assert np.allclose(y, [1.0 + 0.5 * 3.0 * 2.0, 1.0])
    L, g = OM.loss_and_grad(p, X, np.array([4.0, 1.0]))
    # r = [0, 0] -> zero loss and gradient
    assert L == 0.0 and np.all(g == 0.0)


def test_features_definitions_on_a_rank_one_block():
    x = np.linspace(1.0, 2.0, 20)
    y = np.linspace(-1.0, 3.0, 12)
    a = np.outer(x, y)
    f = OM.sketch_features(a, seed=3, index=0)
    fro = np.linalg.norm(a)
    assert abs(f[2] - math.log10(fro)) < 1e-12
    # rank one: A^T A g = sigma^2 (v^T g) v and A g = sigma (v^T g) u, so every ratio
    # ||A^T A g||^2 / (||A g||^2 ||A||_F^2) equals 1 and the stable-rank estimate is 1
    assert abs(f[9]) < 1e-12 and abs(f[10]) < 1e-12 and abs(f[11]) < 1e-12
    assert abs(f[14]) < 1e-12
    assert f[0] == 20 / 256 and f[1] == 12 / 256


def test_workload4_blocks_are_kernel_blocks():
    rb = gen.kernel_blocks_3d(n_points=2048, seed_index=3)
    assert rb.batch > 0
    assert set(np.unique(rb.m)) <= {64, 128, 256} and set(np.unique(rb.n)) <= {64, 128, 256}
    a = rb.a64(0)
    assert np.all(a > 0) and np.all(a <= 1.0)


def test_features_closed_forms_on_orthogonal_columns():
    # A = Q diag(d) with orthonormal Q: column norms are d, ||A g||^2 = sum_j d_j^2 g_j^2 and
    # ||A^T A g||^2 = sum_j d_j^4 g_j^2, so every feature has a closed form in d and the sketch G
    # (the first 8 columns of Gaussian stream 2 of the matrix).
    import oracle as O
    m, n, seed, index = 40, 24, 5, 3
    q, _ = np.linalg.qr(np.random.default_rng(9).standard_normal((m, n)))
    d = np.logspace(0.5, -3, n)[np.random.default_rng(2).permutation(n)]
    a = q * d
    f = OM.sketch_features(a, seed=seed, index=index)
    G = O.omega(seed, index, 2, n, 0, 8)
    fro2 = float((d * d).sum())
    r = d / math.sqrt(fro2)
    lr = np.log10(r)
    yy = ((d[:, None] * G) ** 2).sum(0)
    ww = ((d[:, None] ** 2 * G) ** 2).sum(0)
    y = yy / fro2
    w = ww / (yy * fro2)
    top = n // 8
    want = [m / 256, n / 256, 0.5 * math.log10(fro2), lr.max(), lr.min(), lr.mean(), lr.std(),
            math.log10(y.mean()), y.std() / y.mean(), math.log10(w.mean()), math.log10(w.max()),
            math.log10(w.min()), math.log10(y.max()), math.log10(y.min()),
            math.log10(fro2 / (ww / yy).max()), np.sort(d * d)[-top:].sum() / fro2]
    assert np.abs(f - np.array(want)).max() < 1e-12, np.abs(f - np.array(want))
