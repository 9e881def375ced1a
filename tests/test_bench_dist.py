"""Multi-rank host logic of bench.py on CPU (gloo, world size 2).

Frames are sharded across ranks with no data-path collective (weak scaling);
the only exchange is the max of the ranks' timed intervals, and the oracle arm
runs on rank 0 alone.
"""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import torch.distributed as dist

    import bench

    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t = bench.max_over_ranks(1.0 + 3.0 * rank, "cpu")
        v = bench.job_value(world, 1e9, 10, t)
        args = type("A", (), dict(gpus=world, steps=1, warmup=0))()
        ran = None
        if rank != 0:
            # the oracle arm returns at once on ranks other than 0
            ran = bench.run_reference(args)
        dist.barrier()
        q.put((rank, t, v, ran))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_weak_scaling_value_gloo():
    import torch.multiprocessing as mp

    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
    res = sorted(q.get(timeout=10) for _ in range(world))
    for rank, t, v, ran in res:
        assert t == pytest.approx(4.0)  # slowest rank's interval on every rank
        assert v == pytest.approx(world * 1e9 * 10 / 4.0 / 1e9)
        assert ran is None


def test_single_process_max_is_identity():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.max_over_ranks(2.5, "cpu") == 2.5
    assert bench.job_value(1, 5e9, 2, 1.0) == pytest.approx(10.0)
