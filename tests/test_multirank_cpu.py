"""The multi-GPU form is replicas only: each rank runs the whole forward on
its own GPU with no data-path collective, and bench.py's timing takes a
barrier and the maximum over ranks.  That host-side logic runs here on two
gloo ranks on the CPU."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        bench.barrier(world)
        ms = 10.0 + 5.0 * rank  # rank 1 is the slower replica
        ms_max = bench.max_over_ranks(world, ms)
        rate = bench.whole_job_rate(world, 1e14, 20, ms_max)
        bench.barrier(world)
        q.put((rank, ms_max, rate))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_the_slowest_time_and_the_job_rate():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
    assert all(p.exitcode == 0 for p in procs)
    got = sorted(q.get(timeout=5) for _ in range(world))
    for rank, ms_max, rate in got:
        assert ms_max == 15.0
        # two replicas of 20 steps of 1e14 units each within 15 ms
        assert rate == pytest.approx(2 * 1e14 * 20 / 0.015)


def test_single_rank_needs_no_process_group():
    assert bench.max_over_ranks(1, 3.5) == 3.5
    assert bench.whole_job_rate(1, 1e14, 10, 2.0) == pytest.approx(5e17)
