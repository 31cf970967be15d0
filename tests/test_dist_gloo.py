"""The multi-process path of bench.py on CPU: two gloo ranks on 127.0.0.1.
Each rank reports its own time; the line uses the slowest rank's time and the
units of all ranks (replicas: one process per GPU, no data-path collective)."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ws, r, local = bench._dist()
    times = [1.0 + rank, 10.0 - rank]          # this rank's step and e2e times
    got = bench.max_over_ranks(times, dist, device="cpu")
    rate = bench.whole_job_rate(1000.0, ws, got[0])
    dist.barrier()
    dist.destroy_process_group()
    q.put((r, ws, local, got, rate))


def test_two_gloo_ranks_reduce_to_the_slowest():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r, (rank, ws, local, got, rate) in enumerate(out):
        assert (rank, ws, local) == (r, 2, r)
        assert got == [2.0, 10.0]                 # max of (1, 2) and of (10, 9)
        assert rate == pytest.approx(1000.0 * 2 / 2.0)


def test_single_process_is_identity():
    assert bench.max_over_ranks([3.0, 4.0], None) == [3.0, 4.0]
    assert bench.whole_job_rate(10.0, 1, 2.0) == 5.0
