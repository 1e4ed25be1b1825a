"""The multi-rank path on the CPU (gloo, world size 2): every matrix is independent, so ranks shard
the batch with no data-path collective; the only collectives are the barrier and the
max-over-ranks reduction of the elapsed time that bench.py uses.  These tests check that the
rank-sharded inputs are exactly the single-process batch split in two (weak scaling: each rank
factors its own, distinct matrices) and that the timing reduction and the whole-job value behave
as the bench computes them."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import sys
    sys.path.insert(0, os.path.join(os.path.dirname(os.path.abspath(__file__)), ".."))
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import torch.distributed as dist
    import bench
    import gen
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        per = 6
        shards = {
            "w0": gen.fp64_32_graded(batch=per, first=rank * per).a,
            "w1": gen.svd64_exp8(batch=per, first=rank * per).a,
            "q1": gen.qr128x32_exp8(batch=per, first=rank * per).a,
            "w2": gen.block512_loguniform(batch=2, first=rank * 2, size=48).a,
        }
        # the bench's timing reduction: every rank reports the slowest rank's time
        t = bench.max_over_ranks(10.0 + 5.0 * rank, world, torch.device("cpu"))
        dist.barrier()
        np.savez(os.path.join(out_dir, f"rank{rank}.npz"), t=np.array([t]), **shards)
    finally:
        dist.destroy_process_group()


def test_two_ranks_shard_the_batch_and_reduce_the_time(tmp_path):
    import torch.multiprocessing as mp
    import gen
    world = 2
    mp.spawn(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    got = [np.load(os.path.join(tmp_path, f"rank{r}.npz")) for r in range(world)]
    # max over ranks: rank 1 reported 15 ms, so both see 15
    assert [float(g["t"][0]) for g in got] == [15.0, 15.0]
    # the shards are the single-process batch, split: no matrix is duplicated or missing
    whole = {"w0": gen.fp64_32_graded(batch=12).a, "w1": gen.svd64_exp8(batch=12).a,
             "q1": gen.qr128x32_exp8(batch=12).a, "w2": gen.block512_loguniform(batch=4, size=48).a}
    for key, full in whole.items():
        joined = np.concatenate([g[key] for g in got])
        assert np.array_equal(joined, full), key
        assert not np.array_equal(got[0][key][0], got[1][key][0]), key
    # whole-job value as the bench forms it: world x per-rank units / the max-reduced step time
    units, ms = 20000, 15.0
    assert world * units / (ms * 1e-3) == pytest.approx(2 * 20000 / 0.015)
