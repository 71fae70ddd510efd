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


def _slab_worker(rank, world, port, q):
    """One rank of a volume split into z-slabs: its slab's parts of ECT, Radon and a hybrid
    transform (the oracle restricted to the slab's vertices stands in for the device's
    result), exchanged by the product's gather in rank order."""
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import numpy as np

    import oracle as O
    from paper_2405_02256_gb300 import slabs, synth

    vol = synth.grf((13, 11, 12), 3.0, seed=420)
    ref = O.critical_tables(vol)
    z0, z1 = slabs.slab_bounds(vol.shape[0], world)[rank]
    lo, hi = z0 * 11 * 12, z1 * 11 * 12
    part = O.CriticalTables(shape=ref.shape)
    for src_i, src_v, dst_i, dst_v in ((ref.lower_idx, ref.lower_val, part.lower_idx, part.lower_val),
                                       (ref.delta_idx, ref.delta_val, part.delta_idx, part.delta_val)):
        for idx, val in zip(src_i, src_v):
            k = (idx >= lo) & (idx < hi)
            dst_i.append(idx[k])
            dst_v.append(val[k])
    part.chi = int(part.lower_val[0].sum())
    dirs = synth.sphere_dirs(20, 421, 0.1, 1.5)
    ect = torch.from_numpy(O.ect_grid(part, dirs, -0.9, 0.9, 17).astype(np.int32))
    rad = torch.from_numpy(O.radon_grid(part, dirs, -0.9, 0.9, 17).astype(np.int32))
    ht = torch.from_numpy(O.hybrid_transform(part, "laplace", dirs)[0])
    g_ect, g_rad, g_ht = (slabs.gather_parts(x) for x in (ect, rad, ht))
    if rank == 0:
        q.put((g_ect.numpy(), g_rad.numpy(), g_ht.numpy(),
               O.ect_grid(ref, dirs, -0.9, 0.9, 17), O.radon_grid(ref, dirs, -0.9, 0.9, 17),
               O.hybrid_transform(ref, "laplace", dirs)))
    dist.barrier()
    dist.destroy_process_group()


def test_slab_exchange_two_ranks():
    """World size 2 over gloo: the gathered slab parts, stacked in rank order, add up to the
    whole volume's ECT and Radon exactly and to its hybrid transform within rounding."""
    import numpy as np

    from paper_2405_02256_gb300 import slabs
    assert slabs.slab_bounds(13, 2) == [(0, 6), (6, 13)]
    assert slabs.slab_bounds(256, 4) == [(0, 64), (64, 128), (128, 192), (192, 256)]
    assert slabs.buffer_planes(0, 6, 13) == (0, 7) and slabs.buffer_planes(6, 13, 13) == (5, 13)
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_slab_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    g_ect, g_rad, g_ht, ect_w, rad_w, (ht_w, norm) = q.get(timeout=180)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert g_ect.shape[0] == 2 and g_ht.shape[0] == 2
    np.testing.assert_array_equal(g_ect.sum(axis=0), ect_w)
    np.testing.assert_array_equal(g_rad.sum(axis=0), rad_w)
    assert np.max(np.abs(g_ht.sum(axis=0) - ht_w) / norm) <= 1e-14
