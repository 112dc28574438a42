"""Seed-partitioned queries (one query split over several GPUs) on one GPU: the parts run one
after another with an in-process threshold exchange, and their merged rows must equal the
unpartitioned query and the oracle.  The multi-process exchange and gather are covered on CPU
by tests/test_multirank.py."""
import pytest

import oracle
import synth

nuri = pytest.importorskip("paper_1807_08888_b300")
from paper_1807_08888_b300 import parallel as par  # noqa: E402

pytestmark = pytest.mark.gpu


def _parts(G, count, run):
    board = par.LocalBoard()
    parts = []
    for idx in range(count):
        par.set_partition(G, idx, count, board)
        parts.append(run())
    par.set_partition(G, 0, 1)
    return parts, board


@pytest.mark.parametrize("which", ["rmat11", "chunglu20k"])
def test_clique_partition_merges_to_the_global_top_k(which):
    g = (synth.rmat(11, 16, seed=5) if which == "rmat11"
         else synth.chung_lu_planted(20000, 20.0, 2.1, 10, 8, 16, seed=5))
    G = nuri.load_graph(g.n, g.src, g.dst)
    for k in (1, 10, 100):
        whole = [(r[0], r[1]) for r in nuri.topk_cliques(G, k)]
        assert whole == [(r[0], tuple(r[1])) for r in oracle.bk_cliques(g, k, False)]
        for count in (2, 3):
            parts, board = _parts(G, count, lambda: nuri.topk_cliques(G, k))
            rows = [[(r[0], r[1]) for r in p] for p in parts]
            assert par.merge_rows(rows, k) == whole, (which, k, count)
            # a part only holds cliques whose seed is its own
            assert sum(p.stats["dequeued"] for p in parts) > 0
    # the partition is cleared: the whole query again
    assert [(r[0], r[1]) for r in nuri.topk_cliques(G, 10)] == \
        [(r[0], tuple(r[1])) for r in oracle.bk_cliques(g, 10, False)]


def test_iso_partition_merges_to_the_global_top_k():
    g = synth.rmat(12, 16, seed=9)
    g.labels = synth.labels_uniform(g.n, 8, seed=109)
    g.weights = synth.weights_uniform(g.n, 0, 1000, seed=209)
    G = nuri.load_graph(g.n, g.src, g.dst, labels=g.labels, weights=g.weights, index_hops=4)
    qs = synth.query_batch(8, seed=12, size_lo=3, size_hi=7, num_labels=8)
    for q in qs:
        for k in (1, 50, 1000):
            whole = [tuple(r) for r in nuri.topk_iso(G, q, k)]
            want = [(r[0], tuple(r[1]), tuple(r[2])) for r in oracle.topk_iso(g, q, k)]
            assert whole == want
            parts, _ = _parts(G, 3, lambda: nuri.topk_iso(G, q, k))
            merged = par.merge_rows([[tuple(r) for r in p] for p in parts], k)
            assert merged == whole, (q, k)
