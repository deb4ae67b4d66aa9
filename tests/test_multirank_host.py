"""The replica (N > 1) path of bench.py with two gloo ranks on the CPU: every
rank solves its own seeded problem (distinct seeds), the job time is the
slowest rank's (max over ranks), the job throughput counts every rank's
unknowns, and the reference arm does its work on rank 0 only."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, queue):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench

    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = [3.0, 5.0][rank]
        slowest = bench.max_over_ranks(ms, dist, "cpu")
        seeds = [None] * world
        dist.all_gather_object(seeds, bench.replica_seed(rank))
        skipped = None
        if rank == 1:  # the reference arm returns without work on other ranks
            skipped = bench.run_reference(None) is None
        dist.barrier()
        queue.put((rank, slowest, seeds, bench.job_throughput(world, 1000, slowest), skipped))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_replica_logic():
    ctx = torch.multiprocessing.get_context("spawn")
    queue = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, queue)) for r in range(2)]
    for p in procs:
        p.start()
    got = dict()
    for _ in procs:
        rank, slowest, seeds, value, skipped = queue.get(timeout=120)
        got[rank] = (slowest, seeds, value, skipped)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank in (0, 1):
        slowest, seeds, value, _ = got[rank]
        assert slowest == 5.0
        assert seeds[0] != seeds[1]
        assert value == pytest.approx(2 * 1000 / 5e-3)
    assert got[1][3] is True
