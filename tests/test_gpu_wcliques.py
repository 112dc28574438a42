"""Parity of the CUDA vertex-weighted clique search (cliques ranked by the sum of their vertex
weights) with the oracle; calls go through the C ABI.  Integer scores and vertex sets: rows
must match bit-exactly."""
import numpy as np
import pytest

import oracle
import synth
from oracle import brute

nuri = pytest.importorskip("paper_1807_08888_b300")
pytestmark = pytest.mark.gpu


def load(g):
    return nuri.load_graph(g.n, g.src, g.dst, weights=g.weights)


def rows(res):
    return [(r[0], r[1]) for r in res]


def orows(g, k, maximal=False):
    return [(r[0], tuple(r[1])) for r in oracle.topk_wcliques(g, k, maximal)]


def _weighted(g, seed, hi):
    g.weights = np.random.default_rng(seed).integers(0, hi + 1, size=g.n).astype(np.int32)
    return g


def test_tiny_graphs_vs_oracle_and_brute():
    rng = np.random.default_rng(2)
    for i in range(80):
        n = int(rng.integers(1, 14))
        g = _weighted(synth.er_small(n, [0.2, 0.5, 0.8][i % 3], seed=2600 + i), i, [3, 60][i % 2])
        G = load(g)
        for maximal in (False, True):
            every = [(s, tuple(c)) for s, c in brute.topk_wcliques(g, 10 ** 9, maximal)]
            for k in (1, 3, 10, 60):
                got = rows(nuri.topk_cliques(G, k, maximal=maximal, weighted=True))
                assert got == every[:k], (g.name, k, maximal)
                assert orows(g, k, maximal) == every[:k]


@pytest.mark.parametrize("n,p", [(100, 0.6), (150, 0.55), (200, 0.5)])
def test_dense_records_split_vs_oracle(n, p):
    # degeneracy above 64: records with more than 64 candidates are split into children
    g = _weighted(synth.er_small(n, p, seed=77), 5, 1000)
    G = load(g)
    assert G.info()["max_out_degree"] > 64 or n == 100
    for k in (1, 10, 100):
        assert rows(nuri.topk_cliques(G, k, weighted=True)) == orows(g, k), k


def test_rmat_vs_oracle():
    g = _weighted(synth.rmat(10, 16, seed=10), 210, 1000)
    G = load(g)
    for k in (1, 10, 100, 1000):
        assert rows(nuri.topk_cliques(G, k, weighted=True)) == orows(g, k), k
    assert rows(nuri.topk_cliques(G, 10, maximal=True, weighted=True)) == orows(g, 10, True)


def test_unit_weights_rank_by_size():
    """With every weight 1 the weighted ranking is the ranking by size: the two CUDA
    searches agree on graphs beyond the oracle's reach (the size search is oracle-checked)."""
    for g in (synth.rmat(12, 16, seed=2),
              synth.chung_lu_planted(20000, 20.0, 2.1, 10, 8, 16, seed=7)):
        g.weights = np.ones(g.n, np.int32)
        G = load(g)
        for k in (1, 50, 500):
            assert rows(nuri.topk_cliques(G, k, weighted=True)) == rows(nuri.topk_cliques(G, k))


def test_ties_restart_batch_and_errors(monkeypatch):
    g = _weighted(synth.er_small(40, 0.4, seed=43), 9, 2)  # few distinct scores: many ties
    G = load(g)
    every = [(s, tuple(c)) for s, c in brute.topk_wcliques(g, 10 ** 9)]
    for k in (1, 5, 20):
        cut = every[k - 1][0]
        assert rows(nuri.topk_cliques(G, k, keep_ties=True, weighted=True)) == \
            [r for r in every if r[0] >= cut]
    # no pruning: the same rows
    assert rows(nuri.topk_cliques(G, 20, no_prune=True, weighted=True)) == every[:20]
    # a tiny result set overflows: the query re-runs from its final threshold
    monkeypatch.setenv("NURI_RESULT_CAP", "8")
    got = nuri.topk_cliques(G, 20, weighted=True)
    monkeypatch.delenv("NURI_RESULT_CAP")
    assert got.stats["restarts"] >= 1 and rows(got) == every[:20]
    # one batch: weighted and by-size requests, several k; each equals its own query
    outs = nuri.topk_batch(G, [("clique", 7, False, False, True), ("clique", 7),
                               ("clique", 20, False, False, True)])
    assert rows(outs[0]) == every[:7] and rows(outs[2]) == every[:20]
    assert rows(outs[1]) == rows(nuri.topk_cliques(G, 7))
    # a graph without weights cannot rank by them
    U = nuri.load_graph(g.n, g.src, g.dst)
    with pytest.raises(nuri.NuriError):
        nuri.topk_cliques(U, 5, weighted=True)


def test_handed_back_records_keep_rows_exact(monkeypatch):
    """A launch output smaller than a round's children: records whose children do not fit are
    handed back whole and redone, and output slots past the granted reservations must not
    bring back records of an earlier launch.  Rows equal the oracle's."""
    g = _weighted(synth.er_small(200, 0.5, seed=77), 5, 1000)
    G = load(g)
    want = {k: orows(g, k) for k in (1, 10, 100)}
    monkeypatch.setenv("NURI_WOUT_CAP", "150")
    for k in (1, 10, 100):
        assert rows(nuri.topk_cliques(G, k, weighted=True)) == want[k], k
    monkeypatch.delenv("NURI_WOUT_CAP")
