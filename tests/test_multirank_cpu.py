"""The multi-rank aggregation of bench.py on CPU: two gloo ranks (127.0.0.1), each with its own
timed-region length; the job rate uses the slowest rank and counts every rank's steps."""
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
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        dist.barrier()
        local_seconds = 1.0 + rank  # rank 1 is the slowest
        slowest = bench.dist_max(local_seconds, "cpu")
        rate = bench.whole_job_rate(100, world, slowest)
        dist.barrier()
        out[rank] = (slowest, rate, bench.dist_env())
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_rank():
    world = 2
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    for rank in range(world):
        slowest, rate, env = out[rank]
        assert slowest == 2.0
        assert rate == pytest.approx(world * 100 / 2.0)
        assert env == (rank, world, rank)


def test_single_process_is_identity():
    import bench
    assert bench.dist_max(3.5) == 3.5
    assert bench.whole_job_rate(10, 1, 2.0) == 5.0
