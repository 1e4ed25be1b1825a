"""GPU parity for the learned rank predictor: sketch features, forward, gradient and Adam step
against the FP64 oracle, training, and the gain over the plain adaptive randomized SVD."""
import math
import os

import numpy as np
import pytest

import gen
import oracle as O
from oracle import mlp as OM

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bs():
    import paper_1707_05141_gb300 as bs
    bs.build()
    assert torch.cuda.is_available()
    return bs


@pytest.fixture(scope="module")
def kernel_blocks():
    return gen.kernel_blocks_3d(n_points=4096, seed_index=11)


def test_sketch_features_match_oracle(bs, kernel_blocks):
    from paper_1707_05141_gb300 import rank_mlp
    rb = kernel_blocks
    sel = list(range(0, rb.batch, max(1, rb.batch // 24)))[:24]
    flat = torch.from_numpy(rb.flat).cuda()
    f = rank_mlp.features(flat, rb.offset, rb.m, rb.n, seed=77).cpu().numpy().astype(np.float64)
    for b in sel:
        fo = OM.sketch_features(rb.a64(b), 77, b)
        assert np.abs(f[b] - fo).max() <= 2e-4 * max(1.0, np.abs(fo).max()), (b, f[b] - fo)


def test_forward_and_gradient_match_oracle(bs):
    rng = np.random.default_rng(3)
    p = OM.init_params(4) + 0.05 * rng.standard_normal(OM.NPARAMS)
    X = rng.standard_normal((300, 16))
    t = rng.uniform(1.0, 4.0, 300)
    y_o, _ = OM.forward(p, X)
    L_o, g_o = OM.loss_and_grad(p, X, t)
    P = torch.from_numpy(p.astype(np.float32)).cuda()
    Xd = torch.from_numpy(X.astype(np.float32)).cuda()
    td = torch.from_numpy(t.astype(np.float32)).cuda()
    y = torch.empty(300, device="cuda")
    bs.bsvd_mlp_forward(Xd, P, y)
    g = torch.empty(OM.NPARAMS, device="cuda")
    L = torch.empty(1, device="cuda")
    bs.bsvd_mlp_grad(Xd, td, P, g, L)
    torch.cuda.synchronize()
    yh = y.cpu().numpy().astype(np.float64)
    # FP32 forward of an FP32-rounded network: a few ulps of the activations' magnitude
    assert np.abs(yh - y_o).max() <= 1e-4 * max(1.0, np.abs(y_o).max())
    assert abs(float(L.item()) - L_o) <= 1e-4 * max(L_o, 1e-3)
    gh = g.cpu().numpy().astype(np.float64)
    assert np.abs(gh - g_o).max() <= 1e-4 * np.abs(g_o).max()


def test_adam_step_matches_definition(bs):
    rng = np.random.default_rng(9)
    p = rng.standard_normal(OM.NPARAMS).astype(np.float32)
    g = rng.standard_normal(OM.NPARAMS).astype(np.float32)
    m0 = rng.standard_normal(OM.NPARAMS).astype(np.float32) * 0.1
    v0 = rng.uniform(0, 0.1, OM.NPARAMS).astype(np.float32)
    P, G, Mm, Vv = (torch.from_numpy(x.copy()).cuda() for x in (p, g, m0, v0))
    bs.bsvd_mlp_adam(P, G, Mm, Vv, step=3, lr=1e-2)
    torch.cuda.synchronize()
    b1, b2, eps, lr = 0.9, 0.999, 1e-8, 1e-2
    m = b1 * m0.astype(np.float64) + (1 - b1) * g
    v = b2 * v0.astype(np.float64) + (1 - b2) * g.astype(np.float64) ** 2
    ref = p - lr * (m / (1 - b1 ** 3)) / (np.sqrt(v / (1 - b2 ** 3)) + eps)
    assert np.abs(P.cpu().numpy() - ref).max() <= 1e-5


def test_checkpoint_roundtrip(bs, tmp_path):
    from paper_1707_05141_gb300 import rank_mlp
    p = rank_mlp.init_params(5)
    path = os.path.join(tmp_path, "w.bin")
    rank_mlp.save(path, p, {"tol": 1e-5})
    q, hdr = rank_mlp.load(path)
    assert np.array_equal(p, q) and hdr["tol"] == 1e-5 and hdr["nparams"] == OM.NPARAMS
    with open(path, "r+b") as f:
        f.write(b"XXXXXXXX")
    with pytest.raises(ValueError):
        rank_mlp.load(path)


def test_training_learns_and_beats_plain_adaptive(bs):
    """Train on one point set's ranks (plain adaptive), predict on another: fewer sampling rounds
    at the same 1e-5 truncation error."""
    from paper_1707_05141_gb300 import rank_mlp
    train_b = gen.kernel_blocks_3d(n_points=8192, seed_index=21)
    test_b = gen.kernel_blocks_3d(n_points=8192, seed_index=22)
    ft = torch.from_numpy(train_b.flat).cuda()
    fe = torch.from_numpy(test_b.flat).cuda()
    ranks, _ = rank_mlp.plain_adaptive_ranks(ft, train_b.offset, train_b.m, train_b.n, seed=5)
    feats = rank_mlp.features(ft, train_b.offset, train_b.m, train_b.n, seed=6)
    params, hist = rank_mlp.train(feats, ranks, steps=1500, log_every=500)
    assert hist[-1][1] < 0.05, hist                            # log-rank fit well below 1
    plain = bs.rsvd(fe, test_b.offset, test_b.m, test_b.n, rank_hint=None, max_rounds=16, seed=7)
    fe_feats = rank_mlp.features(fe, test_b.offset, test_b.m, test_b.n, seed=6)
    _, hint = rank_mlp.predict(fe_feats, params, margin=2.0, m=test_b.m, n=test_b.n)
    learned = bs.rsvd(fe, test_b.offset, test_b.m, test_b.n, rank_hint=hint, max_rounds=16, seed=7)
    torch.cuda.synchronize()
    r_plain = (plain.info.cpu().numpy() & 0xFF).mean()
    r_learn = (learned.info.cpu().numpy() & 0xFF).mean()
    assert r_learn < 0.7 * r_plain, (r_learn, r_plain)
    # the error gate on a sample of blocks, both methods
    for res in (plain, learned):
        U, S, V = (t.cpu().numpy().astype(np.float64) for t in (res.U, res.S, res.V))
        rk = res.rank.cpu().numpy()
        for b in range(0, test_b.batch, max(1, test_b.batch // 40)):
            a = test_b.a64(b)
            m, n, k = a.shape[0], a.shape[1], int(rk[b])
            u = U[res.off_u[b]:res.off_u[b] + m * k].reshape(k, m).T
            v = V[res.off_v[b]:res.off_v[b] + n * k].reshape(k, n).T
            s = S[res.off_s[b]:res.off_s[b] + k]
            assert np.linalg.norm(a - (u * s) @ v.T) <= 1e-5 * np.linalg.norm(a), b
