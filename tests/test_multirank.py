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


def _partition_rank(rank, world, port, out):
    """One part of a seed-partitioned top-k clique query on CPU: the part's cliques are those
    whose seed (their smallest vertex: the oracle's canonical order) falls in it; the parts
    exchange thresholds through the process group's store (unequal numbers of calls, no
    waiting) and merge their top-k lists with an all-gather."""
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import synth
    from oracle import brute
    from paper_1807_08888_b300 import parallel as par
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        store = dist.distributed_c10d._get_default_store()
        board = par.TauBoard(store, rank, world, tag="cliques")
        results = {}
        for seed, k in ((77, 10), (78, 40)):
            g = synth.er_small(20, 0.5, seed=seed)
            mine = [c for c in brute.all_cliques(g) if par.seed_part(c[0], world) == rank]
            mine.sort(key=lambda c: (-len(c), c))
            top = [(len(c), c) for c in mine[:k]]
            local = top[-1][0] if len(top) >= k else par.INT64_MIN
            for _ in range(1 + 2 * rank):       # parts call the exchange unequal times
                best = board(seed, local)
            dist.barrier()
            best = board(seed, local)           # every part has published by now
            kept = [r for r in top if r[0] >= best]
            results[seed] = (best, par.gather_merge(kept, k), local)
        out.put((rank, results))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_seed_partition_exchange_and_merge_over_two_gloo_ranks():
    sys.path.insert(0, ROOT)
    import oracle
    import synth
    from oracle import brute
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_partition_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=180) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for seed, k in ((77, 10), (78, 40)):
        g = synth.er_small(20, 0.5, seed=seed)
        want = [(s, tuple(c)) for s, c in brute.topk_cliques(g, k)]
        assert want == [(r[0], tuple(r[1])) for r in oracle.topk_cliques(g, k)]
        b0, m0, l0 = got[0][seed]
        b1, m1, l1 = got[1][seed]
        assert b0 == b1 == max(l0, l1)          # the exchanged threshold is the best part's
        assert [(r[0], tuple(r[1])) for r in m0] == want == [(r[0], tuple(r[1])) for r in m1]


def test_local_board_and_merge():
    sys.path.insert(0, ROOT)
    from paper_1807_08888_b300 import parallel as par
    b = par.LocalBoard()
    assert b(0, par.INT64_MIN) == par.INT64_MIN
    assert b(0, 5) == 5 and b(0, 3) == 5 and b(1, 2) == 2
    rows = par.merge_rows([[(3, (1, 2, 3)), (2, (0, 4))], [(3, (0, 5, 6)), (2, (0, 1))]], 3)
    assert rows == [(3, (0, 5, 6)), (3, (1, 2, 3)), (2, (0, 1))]
