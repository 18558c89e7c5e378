"""The multi-GPU form of the benchmark is replicas only (every rank steps its
own fault; the path has no exchange step): the job's time is the slowest
rank's and its rate counts every rank's elements.  The aggregation runs here
as two gloo ranks on the CPU."""
import os
import socket

import pytest


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank: int, world: int, port: int, q) -> None:
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    # rank r took (r + 1) * 0.5 s for its K steps of N elements
    t = bench._max_over_ranks(torch, 0.5 * (rank + 1), world, device="cpu")
    q.put((rank, t, bench._job_rate(world, 4096, 100, t)))
    dist.barrier()
    dist.destroy_process_group()


def test_replica_timing_is_the_slowest_rank_and_counts_every_rank():
    import torch.multiprocessing as mp
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for rank, t, rate in out:
        assert t == pytest.approx(1.0)                  # the slower rank's 1.0 s
        assert rate == pytest.approx(2 * 4096 * 100 / 1.0)
