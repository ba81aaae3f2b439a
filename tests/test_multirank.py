"""The multi-rank bench path on CPU: two gloo ranks, each on its own shard,
reduce to the slowest rank's time and all ranks' queries; the reference arm
runs on rank 0 only; shards draw distinct problems."""
import os
import socket

import numpy as np
import pytest

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    ms = [10.0, 25.0][rank]
    n_q = [100, 300][rank]
    out.put((rank, bench.reduce_over_ranks(dist, ms, n_q, "cpu")))
    dist.barrier()
    dist.destroy_process_group()


def test_reduce_over_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(60)
        assert p.exitcode == 0
    for r in range(2):
        ms, n_all = got[r]
        assert ms == 25.0 and n_all == 400


def test_single_rank_reduce_is_identity():
    assert bench.reduce_over_ranks(None, 7.5, 123, "cpu") == (7.5, 123)


def test_reference_arm_only_on_rank0(capsys):
    class A:
        workload, steps, warmup = 1, 1, 3
    assert bench.run_reference(A(), 1, 2) is None
    assert capsys.readouterr().out == ""


def test_shards_draw_distinct_problems():
    d0, q0, _ = bench.workload(1, shard=0)
    d1, q1, desc1 = bench.workload(1, shard=1)
    assert q0[0].shape == q1[0].shape
    assert not np.array_equal(q0[0], q1[0])
    assert not np.array_equal(d0[0]["cps"], d1[0]["cps"])
    assert "shard 1" in desc1
