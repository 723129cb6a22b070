"""bench.py's multi-GPU path is replicas only (independent problems, no
data-path collective): the whole-job rate is the units of every rank over
the slowest rank's time.  The aggregation runs here on two gloo ranks on the
CPU (127.0.0.1)."""
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
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        units = [100.0, 300.0][rank]
        secs = [1.0, 2.0][rank]
        rate, tot, smax = bench.replica_rate(units, secs, device="cpu")
        mx = bench.reduce_scalar(rank + 5, "max", device="cpu")
        q.put((rank, rate, tot, smax, mx))
    finally:
        dist.destroy_process_group()


def test_replica_rate_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, rate, tot, smax, mx in out:
        assert tot == 400.0 and smax == 2.0 and rate == 200.0 and mx == 6.0


def test_single_process_is_identity():
    import bench
    assert not dist.is_initialized()
    assert bench.replica_rate(10, 2.5, device="cpu") == (4.0, 10.0, 2.5)
