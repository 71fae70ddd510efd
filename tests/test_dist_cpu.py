"""Multi-rank timing of bench.py on CPU with the gloo backend (world size 2).

Each rank times its own replica (weak scaling: no data-path collective); the job time
is the maximum over ranks and the value counts the units of all ranks.
"""
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
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = 100.0 + 50.0 * rank           # rank 1 is the slower one
    job_ms = bench.max_over_ranks(ms, torch.device("cpu"))
    value = bench.whole_job_rate(units_per_rank=1000, world=world, ms=job_ms)
    q.put((rank, job_ms, value))
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_and_weak_scaling_value():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [150.0, 150.0]
    assert all(abs(r[2] - 2000 / 0.150) < 1e-6 for r in res)


def test_single_rank_helpers_without_process_group():
    import bench
    assert bench.max_over_ranks(12.5, torch.device("cpu")) == 12.5
    assert bench.whole_job_rate(10, 1, 1000.0) == 10.0
