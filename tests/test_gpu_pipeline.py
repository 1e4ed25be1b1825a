"""The host-in/host-out pipeline (copies overlapped with the computation, chunk by chunk) gives
the same results, bit for bit, as one direct call on the device."""
import numpy as np
import pytest

import gen

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_chunked_pipeline_matches_direct_call():
    import paper_1707_05141_gb300 as bs
    from paper_1707_05141_gb300.pipeline import ChunkPipeline
    bs.build()
    dev = torch.device("cuda")
    b = gen.svd64_exp8(batch=1000)
    h_a = torch.from_numpy(b.a).pin_memory()
    d_a = h_a.to(dev)
    outs = [torch.empty((1000, 1, 64), device=dev), torch.empty((1000, 64, 64), device=dev),
            torch.empty((1000, 64, 64), device=dev)]
    info = torch.empty(1000, dtype=torch.int32, device=dev)
    # direct: the whole batch in one call
    s, u, v = (torch.empty_like(o) for o in outs)
    bs.batched_svd_jacobi(bs.Batch.uniform(d_a, 64, 64), bs.Batch.uniform(s, 64, 1), bs.Batch.uniform(u, 64, 64),
                          bs.Batch.uniform(v, 64, 64), info)
    torch.cuda.synchronize()
    # pipelined: 4 chunks, host in, host out
    h_out = [torch.zeros(o.shape, dtype=o.dtype).pin_memory() for o in outs]
    d_in = [torch.zeros_like(d_a)]
    chunk_info = torch.empty(1000, dtype=torch.int32, device=dev)

    pipe = ChunkPipeline([h_a], h_out, d_in, outs, lambda c0, c1, di, do, st: None, chunks=4)
    batches = {(c0, c1): (bs.Batch.uniform(d_in[0][c0:c1], 64, 64), bs.Batch.uniform(outs[0][c0:c1], 64, 1),
                          bs.Batch.uniform(outs[1][c0:c1], 64, 64), bs.Batch.uniform(outs[2][c0:c1], 64, 64))
               for c0, c1 in pipe.bounds}

    def compute(c0, c1, di, do, st):
        a, sb, ub, vb = batches[(c0, c1)]
        bs.batched_svd_jacobi(a, sb, ub, vb, chunk_info[c0:c1], stream=st)

    pipe.compute = compute
    assert len(pipe.bounds) == 4
    pipe.run()
    torch.cuda.synchronize()
    assert torch.equal(chunk_info, info)
    for h, d in zip(h_out, (s, u, v)):
        assert torch.equal(h, d.cpu())


def test_pipeline_rejects_pageable_host_buffers():
    from paper_1707_05141_gb300.pipeline import ChunkPipeline
    dev = torch.device("cuda")
    h = torch.zeros((8, 4))
    with pytest.raises(ValueError):
        ChunkPipeline([h], [h], [h.to(dev)], [h.to(dev)], lambda *a: None)
