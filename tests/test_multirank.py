"""Multi-rank host logic of bench.py on CPU with gloo (world size 2): the
whole-job value divides the queries of all ranks by the slowest rank's step
time; replicas share no data-path collective."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = [10.0, 25.0][rank]
    e2e = [12.0, 20.0][rank]
    q = [1000, 3000][rank]
    r = bench.aggregate(ms, e2e, q, "cpu")
    out[rank] = (r["ms"], r["e2e_ms"], r["queries"], r["value"])
    dist.destroy_process_group()


def test_aggregate_two_ranks_gloo():
    world = 2
    mgr = mp.get_context("spawn").Manager()   # no fork of a process that has threads
    out = mgr.dict()
    mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    for r in range(world):
        ms, e2e, q, v = out[r]
        assert ms == 25.0 and e2e == 20.0 and q == 4000.0
        assert v == pytest.approx(4000.0 / 0.025)


def test_aggregate_single_process():
    import bench
    r = bench.aggregate(5.0, 6.0, 100)
    assert r["value"] == pytest.approx(100 / 0.005)
