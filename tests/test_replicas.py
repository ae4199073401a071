"""The N > 1 benchmark path runs independent replicas (no data-path collective);
its only exchange is the max-over-ranks of the timed region, checked here with
two gloo ranks on the CPU."""
import os
import socket
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sys.path.insert(0, ROOT)
    import bench
    t_local = 2.0 + rank                 # rank 1 is the slow one
    value, t = bench.whole_job_rate(t_local, steps=3, world=world, device="cpu")
    out[rank] = (value, t)
    dist.barrier()
    dist.destroy_process_group()


def test_replica_rate_uses_the_slowest_rank():
    world = 2
    port = _free_port()
    with mp.get_context("spawn").Manager() as mgr:   # no fork of a threaded process
        out = mgr.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        value, t = res[r]
        assert t == pytest.approx(3.0)
        assert value == pytest.approx(3 * world / 3.0)


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    value, t = bench.whole_job_rate(4.0, steps=2, world=1)
    assert (value, t) == (0.5, 4.0)
