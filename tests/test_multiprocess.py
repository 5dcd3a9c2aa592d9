"""The multi-GPU bench path on CPU: two gloo ranks, each with its own cloud (weak scaling); the
job time is the slowest rank's and the units are summed.  No GPU and no solver data exchange."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch.distributed as dist

    import bench
    from synth import cloud_mid

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    cl = cloud_mid(seed=bench.rank_seed(rank), nw=500)
    times = [10.0 + rank, 20.0 - rank, 5.0]
    (t0, t1, t2), units = bench.aggregate_over_ranks(times, cl.n_unknowns, "cpu", world)
    out[rank] = (t0, t1, t2, units, cl.n_unknowns, float(cl.centres[0, 0]))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_aggregation_is_weak_scaling():
    world = 2
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    r0, r1 = out[0], out[1]
    # every rank sees the same job numbers: max of each time, sum of units
    assert r0[:4] == r1[:4]
    assert r0[0] == 11.0 and r0[1] == 20.0 and r0[2] == 5.0
    assert r0[3] == r0[4] + r1[4]
    # the ranks solved different clouds
    assert r0[5] != r1[5]
