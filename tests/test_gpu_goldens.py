"""The CUDA path against oracle-written expected results on the workloads' own shapes (needs
a GPU; calls go through the C ABI).

The expected rows were written once by tests/golden/make_goldens.py, which runs only the
oracle (Bron-Kerbosch / Algorithm 1 for cliques, Algorithm 1 with the isomorphism functions,
Algorithm 2 for patterns) on the seeded inputs; each file records the SHA-256 of its input so a
generator change cannot pass silently.  Integer results: equality, row for row.
"""
import json
import os
import sys

import pytest

import synth

nuri = pytest.importorskip("paper_1807_08888_b300")
pytestmark = pytest.mark.gpu

GOLD = os.path.join(os.path.dirname(__file__), "golden")
sys.path.insert(0, GOLD)
from make_goldens import (CHUNGLU_CASES, CLIQUE_CASES, chunglu_graph, clique_graph,  # noqa: E402
                          row_digest, wclique_graph)


def _golden(name):
    path = os.path.join(GOLD, name)
    if not os.path.exists(path):
        pytest.fail(f"missing golden {name}: run tests/golden/make_goldens.py")
    with open(path) as f:
        return json.load(f)


@pytest.mark.parametrize("case", sorted(CLIQUE_CASES))
def test_cliques_eight_word_tier_vs_bron_kerbosch(case):
    """Graphs whose degeneracy-ordered candidate sets pass 256 vertices: their records are
    searched on 8-word adjacency rows (257..512 candidates) by the task kernel.  Every k of
    the all-cliques ranking and the maximal ranking equal the oracle's rows."""
    d = _golden(f"cliques_{case}.json")
    g = clique_graph(case)
    assert g.sha256() == d["sha256_graph"], "generator changed: rewrite the golden"
    G = nuri.load_graph(g.n, g.src, g.dst)
    assert G.info()["max_out_degree"] > 256
    allr = [(r[0], tuple(r[1])) for r in d["all"]]
    for k in sorted({1, 10, 100, len(allr)}):
        got = nuri.topk_cliques(G, k)
        assert [(r[0], r[1]) for r in got] == allr[:k], (case, k)
        assert got.stats["dense_records"][2] > 0, "no record reached the 8-word tier"
        assert got.stats["tail_launches"] > 0
    maxr = [(r[0], tuple(r[1])) for r in d["maximal"]]
    got = nuri.topk_cliques(G, len(maxr), maximal=True)
    assert [(r[0], r[1]) for r in got] == maxr
    # the same search with another task granularity and the tie-aware pruning off
    os.environ["NURI_TASK_SPLIT"] = "24"
    os.environ["NURI_NO_LEX"] = "1"
    try:
        again = nuri.topk_cliques(G, 100)
    finally:
        del os.environ["NURI_TASK_SPLIT"]
        del os.environ["NURI_NO_LEX"]
    assert [(r[0], r[1]) for r in again] == allr[:100]


@pytest.mark.parametrize("case", sorted(CHUNGLU_CASES))
def test_cliques_headline_recipe_vs_bron_kerbosch(case):
    """The headline's own recipe (Chung-Lu power law, mean degree 20, exponent 2.1, 50
    planted cliques of 15..30) at the largest size the oracle finishes: top-100 by size with
    the lexicographic tie-break, row for row, with the autotuned and the default task
    granularity."""
    d = _golden(f"cliques_{case}.json")
    g = chunglu_graph(case)
    assert g.sha256() == d["sha256_graph"]
    G = nuri.load_graph(g.n, g.src, g.dst)
    want = [(r[0], tuple(r[1])) for r in d["all"]]
    for k in (1, 10, 100):
        assert [(r[0], r[1]) for r in nuri.topk_cliques(G, k)] == want[:k], k
    nuri.tune_cliques(G, 100)
    assert [(r[0], r[1]) for r in nuri.topk_cliques(G, 100)] == want
    assert [(r[0], r[1]) for r in nuri.topk_batch(G, [("clique", 100)])[0]] == want


def test_weighted_cliques_rmat11_vs_oracle():
    """Cliques ranked by vertex weight on R-MAT 11 (weights 0..1000): top-100 of Algorithm 1
    with the weighted bound (48 s in the oracle), row for row, one query and in a batch."""
    d = _golden("wcliques_rmat11_top100.json")
    g = wclique_graph()
    assert g.sha256() == d["sha256_graph"]
    G = nuri.load_graph(g.n, g.src, g.dst, weights=g.weights)
    want = [(r[0], tuple(r[1])) for r in d["rows"]]
    for k in (1, 10, 100):
        assert [(r[0], r[1]) for r in nuri.topk_cliques(G, k, weighted=True)] == want[:k], k
    outs = nuri.topk_batch(G, [("clique", 100, False, False, True), ("clique", 7, False, False, True)])
    assert [(r[0], r[1]) for r in outs[0]] == want
    assert [(r[0], r[1]) for r in outs[1]] == want[:7]


def test_iso_rmat20_sixty_four_queries_vs_oracle():
    """The 64 seeded queries of the R-MAT scale-20 workload (4..8 vertices, paths, cycles,
    stars, trees), top-1000 each, in one batched launch: every query's rows equal the
    oracle's (digest of all 1000 rows, plus the first rows and the k-th score in the clear)."""
    d = _golden("iso_rmat20_top1000.json")
    g = synth.workload("rmat20")
    assert g.sha256() == d["sha256_graph"]
    G = nuri.load_graph(g.n, g.src, g.dst, labels=g.labels, weights=g.weights, index_hops=4)
    qs = synth.query_batch(64, seed=1)
    res = nuri.topk_iso_batch(G, qs, [1000] * 64)
    for i, (q, r, want) in enumerate(zip(qs, res, d["queries"])):
        assert want["query"]["edges"] == [list(e) for e in q.edges]
        rows = [(x[0], x[1], x[2]) for x in r]
        assert len(rows) == want["count"], i
        assert [[x[0], list(x[1]), [list(e) for e in x[2]]] for x in rows[:3]] == want["head"], i
        assert (rows[-1][0] if rows else None) == want["kth_score"], i
        assert row_digest(rows) == want["digest"], i
    # one query at a time gives the same rows (a sample: every eighth query)
    for i in range(0, 64, 8):
        alone = nuri.topk_iso(G, qs[i], 1000)
        assert row_digest([(x[0], x[1], x[2]) for x in alone]) == d["queries"][i]["digest"]


def test_patterns_rmat18_zipf_vs_oracle():
    """Top-10 patterns of exactly M edges on the R-MAT scale-18 Zipf-labelled workload:
    supports, label lists and canonical edge lists equal the oracle's rows for M = 1..5 (the
    oracle's M = 5 run took 3.6 hours)."""
    d = _golden("patterns_rmat18z_top10.json")
    g = synth.workload("rmat18z")
    assert g.sha256() == d["sha256_graph"]
    G = nuri.load_graph(g.n, g.src, g.dst, labels=g.labels)
    assert {"1", "2", "3", "4", "5"} <= set(d["M"])
    for M, want in sorted(d["M"].items()):
        got = nuri.topk_patterns(G, int(M), 10)
        assert [[r[0], list(r[1]), [list(e) for e in r[2]]] for r in got] == want["rows"], M
