"""The bench's multi-GPU path (independent replicas, max-over-ranks timing) on CPU with gloo,
world size 2.  The path has no data-path collective; only the barrier and the max reduction of
the timing cross processes."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist

    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    dev = torch.device("cpu")
    bench.replica_barrier(dist, dev)
    ms = [120.0, 150.0][rank]  # per-replica elapsed time
    m = bench.replica_max(dist, ms, dev)
    v = bench.whole_job_value(1e9, 5, world, m)
    out[rank] = (m, v)
    dist.destroy_process_group()


def test_two_replicas_max_time_and_aggregate():
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
        m, v = out[r]
        assert m == 150.0
        assert abs(v - 1e9 * 5 * 2 / 0.150 / 1e9) < 1e-9


def test_single_process_is_identity():
    sys.path.insert(0, ROOT)
    import torch

    import bench

    assert bench.replica_max(None, 3.5, torch.device("cpu")) == 3.5
    assert bench.whole_job_value(2e9, 4, 1, 1000.0) == 8.0
