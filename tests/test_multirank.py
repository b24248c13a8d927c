"""The N-replica aggregation of bench.py (max of the per-rank times, sum of the
per-rank work) on a world of two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t_local = 2.0 if rank == 1 else 1.0       # rank 1 is the slow replica
    value, t = bench.job_rate(t_local, points_per_rank=1000, steps=10, dist=dist, device="cpu")
    q.put((rank, value, t))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_replica():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, value, t in out:
        assert t == 2.0                       # max over ranks
        assert value == 2 * 1000 * 10 / 2.0   # whole-job work over the job time


def test_single_process_rate():
    import bench
    value, t = bench.job_rate(0.5, points_per_rank=100, steps=4)
    assert t == 0.5 and value == 800.0


def _worker_sum(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    sizes = [96 * 512, 512 * 512, 128 * 128, 384 * 96, 256 * 192]
    mine = bench.partition_instances(sizes, world)[rank]
    work = float(sum(sizes[i] for i in mine)) * 10
    t_local = 1.0 + rank                      # rank 1 is the slow one
    value, t, total = bench.job_rate_sum(t_local, work, dist=dist, device="cpu")
    q.put((rank, mine, value, t, total))
    dist.barrier()
    dist.destroy_process_group()


def test_batch_partition_covers_every_instance_once():
    import bench
    sizes = [96 * 512, 512 * 512, 128 * 128, 384 * 96, 256 * 192, 96 * 96, 512 * 384]
    for world in (1, 2, 3, 4, 8):
        parts = bench.partition_instances(sizes, world)
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(sizes)))
        loads = [sum(sizes[i] for i in p) for p in parts]
        # largest-first to the least-loaded rank: no rank exceeds the mean by
        # more than the largest instance
        assert max(loads) <= sum(sizes) / world + max(sizes)
    assert bench.partition_instances(sizes, 1) == [list(range(len(sizes)))]


def test_two_gloo_ranks_sum_their_batch_shares():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker_sum, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    sizes = [96 * 512, 512 * 512, 128 * 128, 384 * 96, 256 * 192]
    assert sorted(out[0][1] + out[1][1]) == list(range(5))
    for rank, mine, value, t, total in out:
        assert t == 2.0
        assert total == float(sum(sizes)) * 10
        assert value == total / 2.0
