"""World-size-2 gloo checks of the multi-rank bench logic (CPU only): the job
time is the max over ranks and the weak-scaling value counts every rank's field."""

import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, ret):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    local_ms = [3.0, 5.5][rank]
    m = bench.max_over_ranks(local_ms)
    ret[rank] = (m, bench.weak_scaling_value(1000, world, m))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_max_and_weak_scaling_value():
    ctx = mp.get_context("spawn")
    ret = ctx.Manager().dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, ret)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for r in range(2):
        m, v = ret[r]
        assert m == 5.5
        assert v == pytest.approx(2 * 1000 / 5.5e-3)


def test_single_process_needs_no_group():
    import bench

    assert bench.max_over_ranks(2.5) == 2.5
    assert bench.weak_scaling_value(10, 1, 1.0) == pytest.approx(1e4)
