"""The N > 1 path of bench.py on CPU: replicas on two gloo ranks (no GPU).  Each rank runs its
own replica; the whole-job line takes the slowest rank's time and the units of all ranks."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = [1200.0, 1500.0][rank]      # per-rank timed region
        units = [3.0e9, 2.0e9][rank]     # per-rank expansions
        out.put((rank,) + bench.combine_ranks(ms, units, dist, device="cpu"))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_replicas_aggregate_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, units in got:
        assert ms == 1500.0 and units == 5.0e9  # max time, summed units, on every rank


def test_single_process_passes_through():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.combine_ranks(10.0, 7.0) == (10.0, 7.0)
