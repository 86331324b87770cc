"""Multi-rank host logic of bench.py (replicas: slowest rank's time, every
rank's bytes), exercised with two gloo ranks on the CPU."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_ms = [1000.0, 1500.0][rank]
    local_bytes = [2.0e9, 3.0e9][rank]
    max_ms, gbs = bench.aggregate(local_ms, local_bytes, dist)
    out[rank] = (max_ms, gbs)
    dist.barrier()
    dist.destroy_process_group()


def test_aggregate_two_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    for r in range(2):
        max_ms, gbs = out[r]
        assert max_ms == 1500.0
        assert abs(gbs - 5.0e9 / 1.5 / 1e9) < 1e-9


def test_aggregate_single_rank():
    sys.path.insert(0, ROOT)
    import bench
    max_ms, gbs = bench.aggregate(500.0, 1.0e9, None)
    assert max_ms == 500.0 and abs(gbs - 2.0) < 1e-12
