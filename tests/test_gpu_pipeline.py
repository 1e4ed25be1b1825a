"""The host-in/host-out entry points (bsvd_host_svd, bsvd_host_qr: copies overlapped with the
computation, chunk by chunk) give the same results, bit for bit, as one direct call on the device:
every matrix is computed by the same kernel whatever chunk it falls in."""
import numpy as np
import pytest

import gen

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bs():
    import paper_1707_05141_gb300 as bs
    bs.build()
    assert torch.cuda.is_available()
    return bs


@pytest.mark.parametrize("chunks,pinned", [(1, True), (4, True), (7, True), (3, False)])
def test_host_svd_matches_direct_call(bs, chunks, pinned):
    dev = torch.device("cuda")
    b = gen.svd64_exp8(batch=1000)
    h_a = torch.from_numpy(b.a)
    if pinned:
        h_a = h_a.pin_memory()
    d_a = h_a.to(dev)
    u0, s0, v0, i0, _ = bs.svd(d_a)
    mk = lambda *shape, dt=torch.float32: (torch.zeros(shape, dtype=dt).pin_memory() if pinned
                                           else torch.zeros(shape, dtype=dt))
    s, u, v, info = mk(1000, 64), mk(1000, 64, 64), mk(1000, 64, 64), mk(1000, dt=torch.int32)
    ws = torch.empty(bs.host_svd_workspace(bs.F32, 1000, 64, 64), dtype=torch.uint8, device=dev)
    bs.host_svd(h_a, s, u, v, info, chunks=chunks, workspace=ws)
    torch.cuda.synchronize()
    assert torch.equal(info, i0.cpu())
    assert torch.equal(s, s0.cpu().reshape(1000, 64)) and torch.equal(u, u0.cpu()) and torch.equal(v, v0.cpu())


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_host_qr_matches_direct_call(bs, dtype):
    dev = torch.device("cuda")
    b = gen.qr128x32_exp8(batch=300) if dtype == np.float32 else gen.fp64_32_graded(batch=300)
    h_a = torch.from_numpy(b.a).pin_memory()
    q0, r0, i0 = bs.qr(h_a.to(dev))
    bsz, n, m = h_a.shape
    q = torch.zeros((bsz, n, m), dtype=h_a.dtype).pin_memory()
    r = torch.zeros((bsz, n, n), dtype=h_a.dtype).pin_memory()
    info = torch.zeros(bsz, dtype=torch.int32).pin_memory()
    code = bs.F32 if dtype == np.float32 else bs.F64
    ws = torch.empty(bs.host_qr_workspace(code, bsz, m, n), dtype=torch.uint8, device=dev)
    bs.host_qr(h_a, q, r, info, chunks=5, workspace=ws)
    torch.cuda.synchronize()
    assert torch.equal(info, i0.cpu()) and torch.equal(q, q0.cpu()) and torch.equal(r, r0.cpu())


def test_host_entries_refuse_device_tensors_and_short_workspaces(bs):
    dev = torch.device("cuda")
    a = torch.zeros((4, 8, 8))
    s = torch.zeros((4, 8))
    with pytest.raises(ValueError):
        bs.host_svd(a.to(dev), s, workspace=torch.empty(1 << 20, dtype=torch.uint8, device=dev))
    with pytest.raises(bs.BsvdError) as e:
        bs.host_svd(a, s, workspace=torch.empty(16, dtype=torch.uint8, device=dev))
    assert e.value.code == bs.ERR_WORKSPACE


def test_host_calls_on_two_streams_at_once(bs):
    """A QR and an SVD host call enqueued on two streams without a synchronisation in between (the
    bench's end-to-end step): each call's chunks take their own pair of the library's compute
    streams, and both give the direct calls' results bit for bit."""
    dev = torch.device("cuda")
    bq, bsv = gen.qr128x32_exp8(batch=2000), gen.svd64_exp8(batch=2000)
    hq_a, hs_a = torch.from_numpy(bq.a).pin_memory(), torch.from_numpy(bsv.a).pin_memory()
    q0, r0, _ = bs.qr(hq_a.to(dev))
    u0, s0, v0, _, _ = bs.svd(hs_a.to(dev))
    torch.cuda.synchronize()
    pin = lambda *shape: torch.zeros(shape, dtype=torch.float32).pin_memory()
    q, r = pin(2000, 32, 128), pin(2000, 32, 32)
    s, u, v = pin(2000, 64), pin(2000, 64, 64), pin(2000, 64, 64)
    ws_q = torch.empty(bs.host_qr_workspace(bs.F32, 2000, 128, 32), dtype=torch.uint8, device=dev)
    ws_s = torch.empty(bs.host_svd_workspace(bs.F32, 2000, 64, 64), dtype=torch.uint8, device=dev)
    main, side = torch.cuda.current_stream(), torch.cuda.Stream()
    for _ in range(3):  # repeated: the calls alternate over the compute-stream pairs
        side.wait_stream(main)
        bs.host_qr(hq_a, q, r, chunks=5, workspace=ws_q, stream=side)
        bs.host_svd(hs_a, s, u, v, chunks=8, workspace=ws_s, stream=main)
        main.wait_stream(side)
    torch.cuda.synchronize()
    assert torch.equal(q, q0.cpu()) and torch.equal(r, r0.cpu())
    assert torch.equal(s, s0.cpu().reshape(2000, 64)) and torch.equal(u, u0.cpu()) and torch.equal(v, v0.cpu())
