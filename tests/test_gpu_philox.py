"""GPU parity: the sampling generator (Philox4x32-10 + Box-Muller, Algorithm 4's Omega) word for word.

Integer work is compared bit for bit: the device's Philox words equal the published known-answer
vectors (Salmon et al., SC'11; ``tests/golden/``) and the oracle's independent implementation on
thousands of counters.  The Gaussians are compared with the oracle's FP64 Box-Muller on the same
words: the FP64 device samples to a few ulps, the FP32 ones within FP32 evaluation of
z = sqrt(-2 ln u_a) (cos, sin)(2 pi u_b): u_a rounded to FP32 (two roundings) moves -2 ln u_a by up to
4 u32 in absolute terms, so r by up to 4 u32 / (2 r) + (a few ulps of r), and the angle by a few
ulps of 2 pi.
"""
import math
import os

import numpy as np
import pytest

import oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24


@pytest.fixture(scope="module")
def bs():
    import paper_1707_05141_gb300 as bs
    bs.build()
    assert torch.cuda.is_available()
    return bs


def _kat(golden_dir):
    rows = []
    with open(os.path.join(golden_dir, "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            w = [int(x, 16) for x in line.split()]
            rows.append((w[0:4], w[4:6], w[6:10]))
    return rows


def test_device_philox_known_answers(bs, golden_dir):
    for ctr, key, out in _kat(golden_dir):
        seed = key[0] | (key[1] << 32)
        words, _, _ = bs.philox_gauss([ctr], seed)
        got = [int(x) & 0xFFFFFFFF for x in words.cpu().numpy()[0]]
        assert got == out, (ctr, key, [hex(x) for x in got])


def _counters(n, seed):
    rng = np.random.default_rng(seed)
    c = rng.integers(0, 2 ** 32, size=(n, 4), dtype=np.uint64)
    c[:8] = [[0, 0, 0, 0], [1, 0, 0, 0], [0, 1, 0, 0], [0, 0, 1, 0], [0, 0, 0, 1],
             [2 ** 32 - 1] * 4, [63, 255, 16383, 1], [5, 7, 12345, 2]]
    return c


def test_device_philox_words_equal_the_oracle(bs):
    seeds = [0, 1707, 20260301, 0xDEADBEEFCAFEF00D]
    for seed in seeds:
        c = _counters(2048, seed & 0xFFFF)
        words, _, _ = bs.philox_gauss(c, seed)
        w = words.cpu().numpy().view(np.uint32)
        key = [seed & 0xFFFFFFFF, seed >> 32]
        for i in range(c.shape[0]):
            want = O.philox4x32_10([int(x) for x in c[i]], key)
            assert np.array_equal(w[i], want), (seed, i)


def test_device_gaussians_match_the_oracle(bs):
    for seed in (1707, 20260301, 0x123456789ABCDEF):
        c = _counters(1024, 3 + (seed & 0xFF))
        c[:, 0] %= 2 ** 30          # row = 4 g + r must fit the generator's 32-bit row index
        words, g32, g64 = bs.philox_gauss(c, seed)
        w = words.cpu().numpy().view(np.uint32).astype(np.float64)
        g32 = g32.cpu().numpy().astype(np.float64)
        g64 = g64.cpu().numpy()
        for i in range(c.shape[0]):
            g, col, idx, tag = (int(x) for x in c[i])
            for r in range(4):
                want = O.gauss(seed, idx, tag, 4 * g + r, col)
                # radius of the Box-Muller pair this row belongs to
                wa = w[i, 2 * (r // 2)]
                rad = math.sqrt(-2.0 * math.log((wa + 0.5) * 2.0 ** -32))
                assert abs(g64[i, r] - want) <= 1e-14 * (1.0 + abs(want)), (i, r, g64[i, r], want)
                tol32 = 8 * U32 * (1.0 + abs(want)) + min(4 * U32 / max(rad, 1e-30), math.sqrt(8 * U32))
                assert abs(g32[i, r] - want) <= tol32, (i, r, g32[i, r], want, tol32)
