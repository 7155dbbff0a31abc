"""The multi-process path of bench.py (one replica per rank, barrier, max-over-
ranks timing, summed work) on CPU with the gloo backend, world size 2."""
import os
import sys
sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import socket

import pytest
import torch
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    import bench
    import torch.distributed as dist
    w, r, _ = bench.dist_setup()
    assert (w, r) == (world, rank)
    bench.barrier(w)
    # rank r processed (r + 1) * 1000 units in (r + 1) seconds
    rate = bench.replica_rate((r + 1) * 1000, float(r + 1), w)
    out[rank] = (rate, bench.max_over_ranks(float(r + 1), w), bench.sum_over_ranks(1.0, w))
    dist.destroy_process_group()


def test_two_rank_replica_accounting():
    world = 2
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    ctx = mp.get_context("spawn")
    procs = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for r in range(world):
        rate, tmax, n = out[r]
        assert n == 2.0
        assert tmax == 2.0
        assert rate == pytest.approx(3000.0 / 2.0)
