"""Parity of the CUDA pattern-mining path (Algorithm 2, MNI support) with the oracle; calls go
through the C ABI.  Supports are exact integers: rows must match bit-exactly."""
import json
import os

import numpy as np
import pytest

import oracle
import synth
from oracle import brute

nuri = pytest.importorskip("paper_1807_08888_b300")
pytestmark = pytest.mark.gpu

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def load(g):
    return nuri.load_graph(g.n, g.src, g.dst, labels=g.labels, weights=g.weights)


def orows(g, M, k):
    return [(r[0], tuple(r[3]), tuple(r[2])) for r in oracle.topk_patterns(g, M, k)]


def grows(res):
    return [(r[0], tuple(r[1]), tuple(r[2])) for r in res]


def test_fig1b_supports():
    d = json.load(open(os.path.join(GOLD, "fig1b_patterns.json")))
    e = np.asarray(d["edges"], np.int32)
    g = synth.Graph(d["n"], e[:, 0].copy(), e[:, 1].copy(),
                    labels=np.asarray(d["labels"], np.uint8))
    G = load(g)
    top = nuri.topk_patterns(G, 2, 1)
    assert top[0][0] == d["top1_2edge"]["f"] and list(top[0][1]) == d["top1_2edge"]["labels"]
    assert grows(nuri.topk_patterns(G, 2, 10)) == orows(g, 2, 10)
    one = nuri.topk_patterns(G, 1, 10)
    assert sorted((r[0], r[1]) for r in one) == [(2, (0, 1)), (3, (1, 1))]


def test_tiny_vs_oracle_and_brute():
    rng = np.random.default_rng(17)
    for i in range(30):
        n = int(rng.integers(3, 10))
        g = synth.er_small(n, [0.3, 0.5][i % 2], seed=800 + i)
        g.labels = rng.integers(0, 2 + i % 2, size=n).astype(np.uint8)
        G = load(g)
        for M in (1, 2, 3):
            for k in (1, 3, 20):
                got = grows(nuri.topk_patterns(G, M, k))
                assert got == orows(g, M, k), (i, M, k)
                if i % 6 == 0:
                    want = brute.topk_patterns(g, M, k)
                    assert [(r[0], brute.code_from_row(len(r[1]), r[1], r[2])) for r in got] == want


@pytest.mark.parametrize("M", [1, 2, 3, 4, 5])
def test_rmat_zipf_vs_oracle(M):
    g = synth.rmat(9, 8, seed=19)
    g.labels = synth.labels_zipf(g.n, 6, 1.2, seed=19)
    G = load(g)
    for k in (1, 10):
        assert grows(nuri.topk_patterns(G, M, k)) == orows(g, M, k), (M, k)


@pytest.mark.parametrize("ef", [8, 16])
def test_five_edge_ranking_vs_oracle(ef):
    """M = 5 (patterns of up to 6 vertices, the largest size of the R-MAT 18 workload) ranked
    against Algorithm 2 on R-MAT 12 with 8 Zipf labels (the oracle takes 3-14 s there)."""
    g = synth.rmat(12, ef, seed=31)
    g.labels = synth.labels_zipf(g.n, 8, 1.2, seed=31)
    G = load(g)
    want = orows(g, 5, 10)
    for k in (1, 4, 10):
        assert grows(nuri.topk_patterns(G, 5, k)) == want[:k], k


def test_reported_supports_are_exact_mni():
    g = synth.rmat(10, 16, seed=23)
    g.labels = synth.labels_zipf(g.n, 8, 1.2, seed=23)
    G = load(g)
    for M in (3, 5):
        for f, labels, edges in nuri.topk_patterns(G, M, 3):
            assert oracle.mni(g, list(labels), list(edges))[0] == f


def test_edge_oriented_expansion_same_rows_more_work():
    """The exhaustive edge-oriented expansion (every connected M-edge subgraph grown one edge
    at a time from one-edge subgraphs and grouped by pattern, the Arabesque way) returns the
    rows of Algorithm 2, and grows far more subgraphs than Algorithm 2 examines candidates."""
    rng = np.random.default_rng(23)
    for i in range(12):
        n = int(rng.integers(3, 10))
        g = synth.er_small(n, [0.3, 0.6][i % 2], seed=850 + i)
        g.labels = rng.integers(0, 2 + i % 2, size=n).astype(np.uint8)
        G = load(g)
        for M in (1, 2, 3, 4):
            for k in (1, 3, 20):
                assert grows(nuri.topk_patterns(G, M, k, edge_oriented=True)) == orows(g, M, k)
    for sc, Ms in ((9, (1, 2, 3, 4)), (7, (5,))):
        g = synth.rmat(sc, 8, seed=19)
        g.labels = synth.labels_zipf(g.n, 6, 1.2, seed=19)
        G = load(g)
        for M in Ms:
            ex = nuri.topk_patterns(G, M, 10, edge_oriented=True)
            assert grows(ex) == orows(g, M, 10), (sc, M)
            pr = nuri.topk_patterns(G, M, 10)
            assert grows(pr) == grows(ex)
            if M >= 3:
                assert ex.stats["expansions"] > pr.stats["expansions"]
    # ties kept alike
    t1 = nuri.topk_patterns(G, 2, 3, keep_ties=True, edge_oriented=True)
    t2 = nuri.topk_patterns(G, 2, 3, keep_ties=True)
    assert grows(t1) == grows(t2)
