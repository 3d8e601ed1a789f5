"""The N>1 host logic of bench.py on two gloo ranks (CPU): each rank runs an
independent replica, the job time is the slowest rank's, and the job value
counts every rank's entries."""
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


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_ms = [4.0, 6.5][rank]
    ms = bench.max_over_ranks(local_ms, dist)
    value = bench.job_gedges(world, 1_000_000_000, ms * 1e-3)
    q.put((rank, ms, value))
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    for rank, ms, value in got:
        assert ms == pytest.approx(6.5)
        assert value == pytest.approx(2 * 1e9 / 6.5e-3 / 1e9)


def test_single_process_needs_no_group():
    import bench
    assert bench.max_over_ranks(3.0, None) == 3.0
    assert bench.job_gedges(1, 4_000_000_000, 0.005) == pytest.approx(800.0)
