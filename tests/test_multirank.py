"""Multi-rank path of bench.py on the CPU (gloo, world size 2): each rank runs one replica,
the step time is the maximum over ranks and the whole-job rate counts every replica."""
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


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = 10.0 + 5.0 * rank  # the slower rank decides the step time
    m = bench.max_over_ranks(ms, world, torch.device("cpu"))
    out[rank] = (m, bench.whole_job_rate(world, m))
    dist.barrier()
    dist.destroy_process_group()


def test_gloo_world2_max_and_rate():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    mp.start_processes(_worker, args=(2, port, out), nprocs=2, join=True, start_method="spawn")
    assert out[0][0] == out[1][0] == 15.0
    assert out[0][1] == pytest.approx(2 * 1000.0 / 15.0)


def test_single_rank_is_identity():
    import bench
    assert bench.max_over_ranks(3.5, 1, torch.device("cpu")) == 3.5
    assert bench.whole_job_rate(1, 500.0) == pytest.approx(2.0)
