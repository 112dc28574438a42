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


@pytest.mark.parametrize("M", [1, 2, 3, 4])
def test_rmat_zipf_vs_oracle(M):
    g = synth.rmat(9, 8, seed=19)
    g.labels = synth.labels_zipf(g.n, 6, 1.2, seed=19)
    G = load(g)
    for k in (1, 10):
        assert grows(nuri.topk_patterns(G, M, k)) == orows(g, M, k), (M, k)


def test_reported_supports_are_exact_mni():
    g = synth.rmat(10, 16, seed=23)
    g.labels = synth.labels_zipf(g.n, 8, 1.2, seed=23)
    G = load(g)
    for M in (3, 5):
        for f, labels, edges in nuri.topk_patterns(G, M, 3):
            assert oracle.mni(g, list(labels), list(edges))[0] == f
