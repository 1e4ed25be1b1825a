"""GPU parity at the benchmark's full sizes, in the launch configuration bench.py times (the slowest
GPU tests).

The workloads are built by bench.py's own workload classes (same generators, sizes, seeds and
calls; the randomized SVDs replayed from their CUDA graphs).  Every output is checked by properties
that hold at any size; sampled matrices are compared with the FP64 oracle one by one.
  * block512: 500 FP32 512 x 512, GRAM, block width 32 -- every sigma against the generator's
    spectrum, two matrices against the oracle's SVD (sigma, orthogonality, residual);
  * rsvd_uneven: 16384 uneven blocks with the rank hint -- the truncation error of 64 sampled
    blocks, and 16 blocks against the oracle's randomized SVD with the same sampling matrix
    (or its SVD for full-rank blocks), the Eckart-Young bound and orthogonality.
"""
import argparse

import numpy as np
import pytest

import oracle as O
from parity import svd_errors

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

EPS = 1e-5
BENCH_SEED = 1707   # the seed bench.py's randomized SVD workloads pass


@pytest.fixture(scope="module")
def bs():
    import paper_1707_05141_gb300 as bs
    bs.build()
    assert torch.cuda.is_available()
    return bs


def check_block512(W, picks):
    """The block workload's outputs after one call: convergence, every sigma against the
    generator, and the matrices ``picks`` against the oracle's SVD."""
    info = W.info.cpu().numpy()
    assert np.all((info > 0) & (info < (1 << 20))), info[(info <= 0) | (info >= (1 << 20))]
    S = W.S.cpu().numpy()[:, 0, :].astype(np.float64)
    # the generator's spectrum: the FP32 rounding of A moves it by ~u ||A||_F (3e-7), far inside 1e-5
    assert np.abs(S - W.sigma).max() <= EPS
    mats = [W.d[b].cpu().numpy().T.astype(np.float64) for b in picks]
    _, So, _, _, _ = O.svd_batch(mats)
    for i, b in enumerate(picks):
        u = W.U[b].cpu().numpy().T.astype(np.float64)
        v = W.V[b].cpu().numpy().T.astype(np.float64)
        e = svd_errors(mats[i], u, S[b], v, So[i])
        assert max(e.values()) <= EPS, (b, e)


def test_block512_full_workload(bs):
    import bench
    W = bench.Block512(argparse.Namespace(block_batch=500, host_inputs=False))
    W.setup(0, torch.device("cuda"))
    W.step(torch.cuda.current_stream())
    torch.cuda.synchronize()
    check_block512(W, [0, 499])


def check_rsvd(W, every, seed=BENCH_SEED):
    """The randomized workload's outputs after one call: flags, the truncation error of 64 sampled
    blocks, and every ``every``-th block against the oracle (randomized SVD with the same sampling
    matrix, or the SVD of a full-rank block), the Eckart-Young bound and orthogonality."""
    rb = W.rb
    info = W.info.cpu().numpy()
    assert np.all(info >= 0)
    assert W.error_sample(64) <= EPS
    U, V, S = (t.cpu().numpy().astype(np.float64) for t in (W.fu, W.fv, W.fs))
    ou, ov, os_ = (np.asarray(x.ptrs.cpu().numpy() - x.ptrs[0].item(), np.int64) // 4 for x in (W.U, W.V, W.S))
    rank, samples = W.rank.cpu().numpy(), W.samples.cpu().numpy()
    for b in range(0, rb.batch, every):
        a = rb.a64(b)
        m, n, k = a.shape[0], a.shape[1], int(rank[b])
        u = U[ou[b]:ou[b] + m * k].reshape(k, m).T
        v = V[ov[b]:ov[b] + n * k].reshape(k, n).T
        s = S[os_[b]:os_[b] + k]
        na = np.linalg.norm(a)
        assert np.linalg.norm(a - (u * s) @ v.T) / na <= EPS, b
        # Eckart-Young: no rank below the optimum reaches eps (one column of slack for rounding)
        assert k >= O.trunc_rank(np.linalg.svd(a, compute_uv=False), na, EPS) - 1, b
        if k:
            assert np.abs(u.T @ u - np.eye(k)).max() <= EPS and np.abs(v.T @ v - np.eye(k)).max() <= EPS, b
            l = int(samples[b])
            if l < min(m, n):
                _, so, _, _ = O.rsvd(a, seed, b, l, 1)
            else:
                _, so, _, _, _ = O.svd(a)
            assert np.abs(s - so[:k]).max() <= EPS * so[0], (b, np.abs(s - so[:k]).max() / so[0])


def test_rsvd_uneven_full_workload(bs):
    import bench
    W = bench.RsvdUneven(argparse.Namespace(rsvd_batch=16384, host_inputs=False))
    W.setup(0, torch.device("cuda"))
    stream = torch.cuda.current_stream()
    for _ in range(3):      # the benchmark's warm-up calls, then the capture it replays
        W.step(stream)
    torch.cuda.synchronize()
    W.capture(stream)
    W.step(stream)          # one replay of the captured call, as the benchmark times it
    torch.cuda.synchronize()
    check_rsvd(W, W.rb.batch // 16)


def test_hmatrix_mlp_full_workload(bs):
    """Workload 4 at full size (32 768 points, about 52 000 kernel blocks): the rank predictor trained
    as the benchmark trains it, its hints fed to the randomized SVD, one replay of the captured
    step.  Every 1/48th block: the truncation error, Eckart-Young, orthogonality and sigma against
    the oracle; the adaptive decisions (rounds, samples) equal the oracle's adaptive range finder
    with the same hint wherever every round's estimate is at least 2x from eps/2."""
    import bench
    W = bench.HmatrixMlp(argparse.Namespace())
    W.setup(0, torch.device("cuda"))
    stream = torch.cuda.current_stream()
    for _ in range(3):
        W.step(stream)
    torch.cuda.synchronize()
    W.capture(stream)
    W.step(stream)
    torch.cuda.synchronize()
    check_rsvd(W, W.rb.batch // 48)
    hint = W.hint_d.cpu().numpy()
    info, samples = W.info.cpu().numpy(), W.samples.cpu().numpy()
    compared = 0
    for b in range(0, W.rb.batch, W.rb.batch // 48):
        r = O.rsvd_adaptive(W.rb.a64(b), BENCH_SEED, b, int(hint[b]), EPS, 8, 1, 16, 160)
        thr = 0.25 * EPS * EPS * r["norm2"]
        if all(e >= 4 * thr or e <= thr / 4 for e in r["est2_round"]):
            compared += 1
            got = (int(info[b]) & 0xff, int(samples[b]))
            assert got == (r["rounds"], r["samples"]), (b, got, r["rounds"], r["samples"])
    assert compared >= 16, compared
