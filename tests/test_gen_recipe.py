"""The generators produce the inputs their recipes state (spectra, shapes, rank hints, kernel
blocks); checked with LAPACK's SVD on the host.  These are the stand-ins for the paper's matrices,
so a change that altered them would silently change every measured workload."""
import math

import numpy as np

import gen


def _sv(a):
    return np.linalg.svd(a, compute_uv=False)


def test_fp64_32_graded_spectrum():
    b = gen.fp64_32_graded(batch=3)
    want = 10.0 ** (-8.0 * np.arange(32) / 31)
    assert np.allclose(b.sigma, want[None, :], rtol=0, atol=0)
    for i in range(3):
        assert np.abs(_sv(b.a64(i)) - want).max() <= 1e-14 * want[0]


def test_svd64_and_qr128_exp8_spectra():
    s64 = gen.svd64_exp8(batch=2)
    q = gen.qr128x32_exp8(batch=2)
    assert (s64.m, s64.n, q.m, q.n) == (64, 64, 128, 32)
    for b, k in ((s64, 64), (q, 32)):
        want = np.exp(-np.arange(k) / 8.0)
        for i in range(2):
            assert np.abs(_sv(b.a64(i)) - want).max() <= 2e-6 * want[0]   # FP32 rounding of A


def test_block512_loguniform_spectrum():
    b = gen.block512_loguniform(batch=2, size=64)
    assert np.all(b.sigma >= 1e-6) and np.all(b.sigma <= 1.0)
    assert np.all(np.diff(b.sigma, axis=1) <= 0)
    for i in range(2):
        assert np.abs(_sv(b.a64(i)) - b.sigma[i]).max() <= 2e-6 * b.sigma[i][0]


def test_rsvd_uneven_blocks_recipe():
    rb = gen.rsvd_uneven_blocks(batch=600)
    shapes = set(zip(rb.m.tolist(), rb.n.tolist()))
    assert shapes == {(m, n) for m in (64, 128, 256) for n in (64, 128, 256)}
    r0 = rb.extra["r0"]
    assert np.all(r0 >= 2.0) and np.all(r0 <= 12.0)
    k = np.minimum(rb.m, rb.n)
    want = np.minimum(np.ceil(r0 * math.log(1e5)).astype(int), k)
    assert np.array_equal(rb.extra["rank_hint"], want)
    full = np.mean(want >= k)
    assert 0.40 <= full <= 0.56, full                                   # 48% expected
    for b in (0, 1, 2):
        s = _sv(rb.a64(b))
        assert np.abs(s - rb.sigma[b][: len(s)]).max() <= 2e-6 * s[0]
        assert np.allclose(rb.sigma[b], np.exp(-np.arange(k[b]) / r0[b]))


def test_kernel_blocks_3d_recipe():
    rb = gen.kernel_blocks_3d(n_points=4096, seed_index=1)
    assert rb.batch > 100
    assert np.all((rb.m >= 64) & (rb.m <= 256) & (rb.n >= 64) & (rb.n <= 256))
    assert all(t != s for t, s in rb.extra["pairs"])                   # admissible: never self blocks
    for b in range(0, rb.batch, max(1, rb.batch // 12)):
        a = rb.a64(b)
        assert np.all(a > 0.0) and np.all(a <= 1.0)                     # exp(-|x - y| / 0.1)
        s = _sv(a)
        tail = np.sqrt(np.cumsum((s ** 2)[::-1])[::-1])
        rank = int(np.argmax(tail <= 1e-5 * np.linalg.norm(a))) if np.any(tail <= 1e-5 * np.linalg.norm(a)) else len(s)
        assert 2 <= rank <= 40, (b, rank)                               # numerically low rank


def test_admissibility_closed_form():
    # unit cubes with a gap g along x: diameters sqrt(3), distance g -> admissible iff sqrt(3) <= eta g
    lo, hi = np.zeros(3), np.ones(3)
    for g, eta, want in [(2.0, 1.1, True), (1.5, 1.1, False), (1.6, 1.1, True), (1.55, 1.1, False),
                         (1.7321, 1.0, True), (1.732, 1.0, False)]:
        a = [0, 0, lo, hi, None]
        b = [0, 0, lo + np.array([1.0 + g, 0, 0]), hi + np.array([1.0 + g, 0, 0]), None]
        assert gen._admissible(a, b, eta) == want, (g, eta)
    # touching boxes are never admissible; a box is never admissible with itself
    a = [0, 0, lo, hi, None]
    assert not gen._admissible(a, [0, 0, lo + np.array([1.0, 0, 0]), hi + np.array([1.0, 0, 0]), None], 10.0)
    assert not gen._admissible(a, a, 10.0)


def test_kd_tree_partitions_with_median_splits():
    pts = gen.uniforms(4, 0, gen.TAG_MISC, 3 * 1000).reshape(1000, 3)
    perm, nodes = gen._kd_tree(pts, 64)
    assert sorted(perm.tolist()) == list(range(1000))
    for s, e, lo, hi, ch in nodes:
        p = pts[perm[s:e]]
        assert np.all(p >= lo) and np.all(p <= hi)
        if ch is None:
            assert e - s <= 64
        else:
            a, b = nodes[ch[0]], nodes[ch[1]]
            assert (a[0], a[1], b[0], b[1]) == (s, (s + e) // 2, (s + e) // 2, e)   # median: equal halves
            d = int(np.argmax(hi - lo))                                               # split along the widest side
            assert pts[perm[a[0]:a[1]], d].max() <= pts[perm[b[0]:b[1]], d].min()
