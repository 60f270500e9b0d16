"""The N > 1 benchmark path on CPU: two gloo ranks, each timing its own problem.

Every rank solves its own contour (weak scaling); the only exchange is the max-over-ranks
reduction of the elapsed time, and the reference arm runs on rank 0 alone.
"""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    os.environ["RANK"] = str(rank)
    os.environ["WORLD_SIZE"] = str(world)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    elapsed, value = bench.aggregate(1.0 + rank, steps=4, world=world, device="cpu")
    class A:
        seed = 0
        steps = 1
        warmup = 3
    # the reference arm (the CPU oracle) runs on rank 0 only: every other rank returns at once,
    # before building a workload or timing anything
    import time
    t0 = time.perf_counter()
    res = bench.reference_arm(A()) if rank != 0 else None
    out[rank] = (elapsed, value, res is None, time.perf_counter() - t0)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_aggregate_max_time():
    world = 2
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        elapsed, value, ok, seconds = res[rank]
        assert elapsed == 2.0                    # max over ranks
        assert value == pytest.approx(4 * world / 2.0)
        assert ok                                # non-zero ranks print nothing
        assert seconds < 1.0                     # and do no reference work
