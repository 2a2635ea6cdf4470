"""The bench's multi-rank host logic on CPU with gloo (world size 2).

Multi-GPU runs are replicas (the single-GPU product does not shard): every
rank times the same workload, the job's time is the slowest rank's, and the
reported value is all ranks' useful flops over that time.
"""
import os
import sys

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    secs = 1.0 + rank                      # rank 1 is the slower one
    t = bench.max_over_ranks(secs, world)
    bench.barrier(world)
    v = bench.aggregate_value(2.0e12, world, 5, t)
    q.put((rank, t, v))
    dist.destroy_process_group()


def test_replicas_take_max_time_and_sum_work():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + (os.getpid() % 1000)
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    out = [q.get(timeout=120) for _ in ps]
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, v in out:
        assert t == 2.0
        assert v == pytest.approx(2.0e12 * 2 * 5 / 2.0 / 1e12)
