"""The multi-GPU path of bench.py (replicas over k, max-over-ranks timing) with two
gloo ranks on CPU: every rank gets distinct k values of the same distribution, and
the timing reduction returns the slowest rank."""
import os
import socket

import numpy as np
import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import sys
    import torch.distributed as dist
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    import workloads as wl
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    k = bench.rank_units(wl.mixed_1024(N=32, nk=16).k, rank, world)
    slowest = bench.allreduce_max(10.0 + rank, dist)
    out[rank] = (k, slowest)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_get_distinct_units_and_the_slowest_time():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    world, port = 2, _free_port()
    with ctx.Manager() as mgr:
        out = mgr.dict()
        procs = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(timeout=120)
            assert p.exitcode == 0
        k0, t0 = out[0]
        k1, t1 = out[1]
    assert t0 == t1 == 11.0                         # max over ranks
    assert k0.shape == k1.shape == (16,)
    np.testing.assert_allclose(np.abs(k0), np.abs(k1), rtol=1e-15)   # same |k| distribution
    assert np.min(np.abs(k0[:, None] - k1[None, :])) > 1e-6         # distinct units
