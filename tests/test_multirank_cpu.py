"""The multi-GPU path of bench.py is replicas only: every rank runs its own instance and the
job's throughput is every rank's particles over the slowest rank's time.  Its host logic is
checked here with world_size 2 on the gloo backend (CPU, no GPU)."""
import os
import socket
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, ws, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    sys.path.insert(0, ROOT)
    import bench

    dist.init_process_group("gloo", rank=rank, world_size=ws)
    local_ms = [100.0, 250.0][rank]          # rank 1 is the slow one
    particles = [1000, 3000][rank]
    ms, value = bench.replica_throughput(local_ms, particles, 10, torch.device("cpu"))
    out[rank] = (ms, value)
    dist.barrier()
    dist.destroy_process_group()


def test_replica_throughput_two_ranks_gloo():
    ws = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    procs = [ctx.Process(target=_rank, args=(r, ws, port, out)) for r in range(ws)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    for r in range(ws):
        ms, value = out[r]
        assert ms == 250.0                                   # the slowest rank's time
        assert value == pytest.approx((1000 + 3000) * 10 / 0.25)   # all ranks' particles


def test_replica_throughput_single_process():
    sys.path.insert(0, ROOT)
    import bench

    ms, value = bench.replica_throughput(200.0, 5000, 4)
    assert ms == 200.0 and value == pytest.approx(5000 * 4 / 0.2)
