"""The multi-rank timing path of bench.py (one independent fit per rank, weak scaling) on
world_size-2 gloo ranks: every rank gets the max of the ranks' durations and the whole-job rate."""

import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    value, t_max = bench.whole_job_value(100.0 + 50.0 * rank, 1e9, world)
    dist.barrier()
    q.put((rank, value, t_max))
    dist.destroy_process_group()


def test_whole_job_value_takes_the_max_over_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    world = 2
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    out = sorted(q.get(timeout=10) for _ in range(world))
    for rank, value, t_max in out:
        assert t_max == pytest.approx(150.0)
        assert value == pytest.approx(world * 1e9 / 0.150)


def test_single_rank_needs_no_process_group():
    import bench

    value, t_max = bench.whole_job_value(200.0, 5e8, 1)
    assert t_max == 200.0 and value == pytest.approx(2.5e9)
