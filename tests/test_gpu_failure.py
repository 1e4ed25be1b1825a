"""GPU: failure detection without a GPU fault.

* The tensor-core Gram's bounded completion wait is made to run out (BSVD_BLOCK_TEST_TIMEOUT: the
  first wait of each pair waits 1 ms on a barrier nothing arrives at); the call must report
  BSVD_INFO_DEVICE_TIMEOUT for every matrix, and the context must stay usable: the same call
  without the flag then gives the correct SVD.
* A NaN or an infinity in the input is reported per matrix (BSVD_INFO_NONFINITE) by every entry
  point, while the other matrices of the batch are unaffected.
* max_sweeps = 1 reports BSVD_INFO_NOT_CONVERGED + 1 (the sweep cap).
"""
import numpy as np
import pytest

import gen
import oracle as O
from parity import svd_errors

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bs():
    import paper_1707_05141_gb300 as bs
    bs.build()
    assert torch.cuda.is_available()
    return bs


def test_tensor_core_wait_timeout_is_reported_and_the_context_survives(bs):
    b = gen.block512_loguniform(batch=3, size=256)
    a = torch.from_numpy(b.a).cuda()
    u, s, v, info, _ = bs.svd_block(a, block_width=32, method=bs.BLOCK_GRAM | bs.BLOCK_TEST_TIMEOUT)
    torch.cuda.synchronize()
    assert list(info.cpu().numpy()) == [bs.INFO_DEVICE_TIMEOUT] * 3
    # the same call without the flag, on the same context
    u, s, v, info, _ = bs.svd_block(a, block_width=32, method=bs.BLOCK_GRAM)
    torch.cuda.synchronize()
    info = info.cpu().numpy()
    assert np.all((info > 0) & (info < (1 << 20))), info
    for i in range(3):
        a64 = b.a64(i)
        _, so, _, _, _ = O.svd(a64)
        e = svd_errors(a64, u[i].cpu().numpy().T.astype(np.float64), s[i].cpu().numpy().astype(np.float64),
                       v[i].cpu().numpy().T.astype(np.float64), so)
        assert max(e.values()) <= 1e-5, (i, e)


def _poisoned(batch_obj, dtype):
    a = batch_obj.a.astype(dtype).copy()
    a[1, 3, 2] = np.nan          # matrix 1: a NaN
    a[2, 0, 0] = np.inf          # matrix 2: an infinity
    return a


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_nonfinite_input_is_flagged_by_every_path(bs, dtype):
    b = gen.uniform_batch(7, 4, 48, 40, np.float64, lambda i: np.exp(-np.arange(40) / 6.0))
    a = torch.from_numpy(_poisoned(b, dtype)).cuda()
    want = [None, bs.INFO_NONFINITE, bs.INFO_NONFINITE, None]
    # register / shared tiers
    for tier in (bs.TIER_REGISTER, bs.TIER_SHARED):
        _, _, _, info, _ = bs.svd(a, tier=tier)
        torch.cuda.synchronize()
        info = info.cpu().numpy()
        assert info[0] >= 0 and info[3] >= 0 and info[1] == info[2] == bs.INFO_NONFINITE, (tier, info)
    # QR
    _, _, info = bs.qr(a)
    torch.cuda.synchronize()
    info = info.cpu().numpy()
    assert info[0] == 0 and info[3] == 0 and info[1] == info[2] == bs.INFO_NONFINITE, info
    # block tier (GRAM and DIRECT)
    for method in (bs.BLOCK_GRAM, bs.BLOCK_DIRECT):
        _, _, _, info, _ = bs.svd_block(a, block_width=16, method=method)
        torch.cuda.synchronize()
        info = info.cpu().numpy()
        assert info[0] > 0 and info[3] > 0 and info[1] == info[2] == bs.INFO_NONFINITE, (method, info)
    # randomized SVD: flagged in the plan, rank 0, nothing computed for those blocks
    flat = a.reshape(-1).contiguous()
    offs = np.arange(4) * 48 * 40
    res = bs.rsvd(flat, offs, [48] * 4, [40] * 4, rank_hint=[8] * 4, tol=1e-4)
    torch.cuda.synchronize()
    info = res.info.cpu().numpy()
    assert info[0] >= 0 and info[3] >= 0 and list(info[1:3]) == [bs.INFO_NONFINITE] * 2, info
    assert list(res.rank.cpu().numpy()[1:3]) == [0, 0]
    for b_, w in enumerate(want):
        if w is None:
            assert int(res.rank.cpu().numpy()[b_]) > 0


def test_sweep_cap_reports_not_converged(bs):
    b = gen.uniform_batch(8, 2, 64, 64, np.float32, lambda i: np.exp(-np.arange(64) / 8.0))
    a = torch.from_numpy(b.a).cuda()
    _, _, _, info, _ = bs.svd(a, max_sweeps=1)
    _, _, _, binfo, _ = bs.svd_block(a, block_width=16, max_sweeps=1)
    torch.cuda.synchronize()
    assert list(info.cpu().numpy()) == [bs.INFO_NOT_CONVERGED + 1] * 2
    assert list(binfo.cpu().numpy()) == [bs.INFO_NOT_CONVERGED + 1] * 2
