"""Parity of the CUDA clique path with the oracle (needs a GPU; calls go through the C ABI).

Cliques are integer set work: results must match bit-exactly (same rows, same order).
"""
import itertools
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


def load(g, **kw):
    return nuri.load_graph(g.n, g.src, g.dst, labels=g.labels, weights=g.weights, **kw)


def rows_oracle(g, k, maximal=False):
    return [(r[0], tuple(r[1])) for r in oracle.topk_cliques(g, k, maximal)]


def test_fig1a():
    d = json.load(open(os.path.join(GOLD, "fig1a_cliques.json")))
    e = np.asarray(d["edges"], np.int32)
    g = synth.Graph(d["n"], e[:, 0].copy(), e[:, 1].copy())
    G = load(g)
    for k, expect in d["topk"].items():
        got = nuri.topk_cliques(G, int(k))
        assert [list(r[1]) for r in got] == expect
    assert [list(r[1]) for r in nuri.topk_cliques(G, 10, maximal=True)] == d["maximal"]
    assert len(nuri.topk_cliques(G, 100)) == d["num_cliques"]


def test_tiny_graphs_vs_oracle_and_brute():
    rng = np.random.default_rng(1)
    for i in range(150):
        n = int(rng.integers(1, 16))
        g = synth.er_small(n, [0.2, 0.5, 0.8][i % 3], seed=2000 + i)
        G = load(g)
        for k in (1, 3, 10, 60):
            for maximal in (False, True):
                want = rows_oracle(g, k, maximal)
                got = [(r[0], r[1]) for r in nuri.topk_cliques(G, k, maximal=maximal)]
                assert got == want, (g.name, k, maximal)
        if i % 10 == 0:
            assert [(r[0], r[1]) for r in nuri.topk_cliques(G, 5)] == \
                [(s, tuple(c)) for s, c in brute.topk_cliques(g, 5)]


_BK_CACHE = {}


def rows_bk(g, key, k, maximal):
    """Top-k from the Bron-Kerbosch oracle (pinned to Algorithm 1 and brute force on tiny
    graphs); the top-1000 list is computed once per graph and sliced."""
    ck = (key, maximal)
    if ck not in _BK_CACHE:
        _BK_CACHE[ck] = [(r[0], tuple(r[1])) for r in oracle.bk_cliques(g, 1000, maximal)]
    return _BK_CACHE[ck][:k]


@pytest.mark.parametrize("scale,ef,seed", [(10, 8, 1), (11, 16, 5), (12, 16, 2)])
@pytest.mark.parametrize("k", [1, 10, 100, 1000])
def test_rmat_vs_oracle(scale, ef, seed, k):
    # power-law rows: exercises the split path (|P| > 64) and the bucketed frontier
    g = synth.rmat(scale, ef, seed=seed)
    G = load(g)
    # maximal mode checks every candidate's maximality with a global adjacency scan: it is
    # exercised here on the smaller cases only
    modes = (False, True) if (scale, k) in ((10, 1), (10, 10), (10, 100), (11, 1), (11, 10),
                                            (12, 1)) else (False,)
    for maximal in modes:
        want = rows_bk(g, (scale, ef, seed), k, maximal)
        got = [(r[0], r[1]) for r in nuri.topk_cliques(G, k, maximal=maximal)]
        assert got == want, (scale, k, maximal)


def test_rmat_small_vs_algorithm1_oracle():
    g = synth.rmat(10, 8, seed=1)
    G = load(g)
    for k in (1, 10, 100):
        assert [(r[0], r[1]) for r in nuri.topk_cliques(G, k)] == rows_oracle(g, k)


def test_planted_er_config():
    g = synth.workload("er2000")
    G = load(g)
    C = sorted(g.planted[0])
    got = nuri.topk_cliques(G, 10)
    want = [tuple(C)] + [tuple(x for x in C if x != C[j]) for j in range(11, 2, -1)]
    assert [r[1] for r in got] == want
    assert [(r[0], r[1]) for r in got] == rows_oracle(g, 10)
    assert [(r[0], r[1]) for r in nuri.topk_cliques(G, 10, maximal=True)] == rows_oracle(g, 10, True)


def test_dense_planted_many_ties():
    # many equal-size cliques: exact lexicographic tie-breaking at the k-th place
    g = synth.er_small(60, 0.5, seed=42)
    G = load(g)
    for k in (1, 7, 50, 333, 5000):
        assert [(r[0], r[1]) for r in nuri.topk_cliques(G, k)] == rows_oracle(g, k)


def test_keep_ties_returns_every_tie():
    g = synth.er_small(40, 0.4, seed=43)
    G = load(g)
    allc = brute.topk_cliques(g, 10 ** 9)
    for k in (1, 5, 20):
        tau = allc[k - 1][0]
        want = [(s, tuple(c)) for s, c in allc if s >= tau]
        got = [(r[0], r[1]) for r in nuri.topk_cliques(G, k, keep_ties=True)]
        assert got == want


def test_no_prune_ablation_same_results_more_work():
    # without pruning every clique is generated: keep the graph's cliques small
    g = synth.er_small(90, 0.25, seed=5)
    G = load(g)
    a = nuri.topk_cliques(G, 20)
    b = nuri.topk_cliques(G, 20, no_prune=True)
    assert [(r[0], r[1]) for r in a] == [(r[0], r[1]) for r in b] == rows_oracle(g, 20)
    assert b.stats["expansions"] >= a.stats["expansions"]


def test_forced_spill_equals_resident(monkeypatch):
    # a small split limit sends most records through the bucketed frontier; a 64-record
    # device frontier then forces spills to pinned host memory and reloads
    g = synth.rmat(11, 16, seed=7)
    G = load(g)
    monkeypatch.setenv("NURI_SPLIT_ABOVE", "4")
    a = nuri.topk_cliques(G, 50)
    b = nuri.topk_cliques(G, 50, frontier_cap=64)
    monkeypatch.delenv("NURI_SPLIT_ABOVE")
    want = [(r[0], tuple(r[1])) for r in oracle.bk_cliques(g, 50, False)]
    assert [(r[0], r[1]) for r in a] == [(r[0], r[1]) for r in b] == want
    assert b.stats["spilled"] > 0 and b.stats["reloaded"] > 0


@pytest.mark.parametrize("split", [2, 5, 16])
def test_split_tier_vs_oracle(monkeypatch, split):
    monkeypatch.setenv("NURI_SPLIT_ABOVE", str(split))
    for g in (synth.rmat(10, 8, seed=1), synth.er_small(120, 0.5, seed=78)):
        G = load(g)
        for k in (1, 10, 100):
            want = [(r[0], tuple(r[1])) for r in oracle.bk_cliques(g, k, False)]
            assert [(r[0], r[1]) for r in nuri.topk_cliques(G, k)] == want, (g.name, k)


@pytest.mark.parametrize("n,p", [(150, 0.55), (200, 0.5), (260, 0.45)])
def test_wide_bitmap_tail_dense_random(n, p):
    # degeneracy above 64: candidate sets of 65..256 vertices go to the 2- and 4-word dense
    # tiers (the 8-word tier, 257..512, is reached by the golden-file tests)
    g = synth.er_small(n, p, seed=77)
    G = load(g)
    assert G.info()["max_out_degree"] > 64
    for k in (1, 10, 100):
        want = [(r[0], tuple(r[1])) for r in oracle.bk_cliques(g, k, False)]
        assert [(r[0], r[1]) for r in nuri.topk_cliques(G, k)] == want, k
    want = [(r[0], tuple(r[1])) for r in oracle.bk_cliques(g, 10, True)]
    assert [(r[0], r[1]) for r in nuri.topk_cliques(G, 10, maximal=True)] == want


def test_result_overflow_restart_is_exact(monkeypatch):
    # a tiny initial result buffer overflows: the query re-runs with the final threshold
    g = synth.er_small(300, 0.08, seed=44)
    G = load(g)
    want = rows_oracle(g, 25)
    monkeypatch.setenv("NURI_RESULT_CAP", "16")
    got = nuri.topk_cliques(G, 25)
    monkeypatch.delenv("NURI_RESULT_CAP")
    assert got.stats["restarts"] >= 1
    assert [(r[0], r[1]) for r in got] == want


def test_result_compaction_keeps_the_top_k(monkeypatch):
    # a small result set fills up across rounds: rows below tau are dropped on the way and the
    # answer is unchanged (compaction, not a re-run, when no single launch overflows it)
    g = synth.chung_lu_planted(20000, 20.0, 2.1, 10, 8, 16, seed=7)
    G = load(g)
    ref = nuri.topk_cliques(G, 50)
    monkeypatch.setenv("NURI_RESULT_CAP", "512")
    got = nuri.topk_cliques(G, 50)
    monkeypatch.delenv("NURI_RESULT_CAP")
    assert [(r[0], r[1]) for r in got] == [(r[0], r[1]) for r in ref]


def test_tie_aware_pruning_keeps_results(monkeypatch):
    # the lexicographic threshold (smallest id of the k-th result among ties) prunes only
    # cliques that rank after k known results: same rows with it switched off
    g = synth.chung_lu_planted(20000, 20.0, 2.1, 10, 8, 16, seed=5)
    G = load(g)
    on = [(r[0], r[1]) for r in nuri.topk_cliques(G, 60)]
    monkeypatch.setenv("NURI_NO_LEX", "1")
    off = [(r[0], r[1]) for r in nuri.topk_cliques(G, 60)]
    monkeypatch.delenv("NURI_NO_LEX")
    assert on == off


def test_tune_cliques_keeps_results():
    # the autotuner times one query per task granularity and keeps the fastest; the answer
    # does not depend on the choice
    g = synth.chung_lu_planted(20000, 20.0, 2.1, 10, 8, 16, seed=3)
    G = load(g)
    ref = [(r[0], r[1]) for r in nuri.topk_cliques(G, 40)]
    chosen, ms = nuri.tune_cliques(G, 40)
    assert chosen in (48, 96, 128, 192) and ms > 0
    assert [(r[0], r[1]) for r in nuri.topk_cliques(G, 40)] == ref


def test_edge_cases():
    # empty graph, isolated vertices, self-loops and duplicate pairs
    G = nuri.load_graph(0, np.zeros(0, np.int32), np.zeros(0, np.int32))
    assert list(nuri.topk_cliques(G, 3)) == []
    G = nuri.load_graph(3, np.zeros(0, np.int32), np.zeros(0, np.int32))
    assert [(r[0], r[1]) for r in nuri.topk_cliques(G, 5)] == [(1, (0,)), (1, (1,)), (1, (2,))]
    src = np.array([0, 1, 1, 2, 2, 0, 3], np.int32)
    dst = np.array([1, 0, 1, 0, 2, 1, 3], np.int32)
    G = nuri.load_graph(4, src, dst)
    info = G.info()
    assert info["num_edges"] == 2 and info["dropped"] == 5
    assert [(r[0], r[1]) for r in nuri.topk_cliques(G, 3)] == [(2, (0, 1)), (2, (0, 2)), (1, (0,))]
    with pytest.raises(nuri.NuriError):
        nuri.load_graph(2, np.array([0], np.int32), np.array([5], np.int32))
    with pytest.raises(nuri.NuriError):
        nuri.topk_cliques(G, 0)


@pytest.mark.parametrize("case", ["er", "clique_path", "rmat16", "rmat17", "chunglu100k"])
def test_peel_order_reaches_the_degeneracy(case):
    # The clique orientation ranks vertices by the batch-peeling (core decomposition) order;
    # its largest out-degree equals the graph's degeneracy, the largest core number, which
    # networkx computes independently.  Graphs of at most 65536 vertices are peeled wholly by
    # the one-CTA tail kernel; the larger ones start in the multi-launch loop and hand a
    # non-empty front over to it (rmat17's hubs also take the tail's whole-CTA row path).
    nx = pytest.importorskip("networkx")
    if case == "er":
        g = synth.er_small(300, 0.1, seed=1)
    elif case == "clique_path":
        c = list(itertools.combinations(range(40), 2)) + [(i, i + 1) for i in range(39, 399)]
        e = np.array(c, np.int32)
        g = synth.Graph(400, e[:, 0].copy(), e[:, 1].copy())
    elif case == "rmat16":
        g = synth.rmat(16, 16, seed=3)
    elif case == "rmat17":
        g = synth.rmat(17, 16, seed=4)
    else:
        g = synth.chung_lu_planted(100_000, 20.0, 2.1, 10, 8, 16, seed=7)
    G = load(g)
    H = nx.Graph()
    H.add_nodes_from(range(g.n))
    H.add_edges_from((int(a), int(b)) for a, b in zip(g.src, g.dst) if a != b)
    expect = max(nx.core_number(H).values()) if g.n else 0
    assert G.info()["max_out_degree"] == expect


def test_clique_limit_is_reported():
    # a 257-clique exceeds the 256-vertex record limit: NURI_ERR_LIMIT, graph still usable
    c = list(range(257))
    e = np.array(list(itertools.combinations(c, 2)), np.int32)
    G = nuri.load_graph(257, e[:, 0].copy(), e[:, 1].copy())
    with pytest.raises(nuri.NuriError) as ei:
        nuri.topk_cliques(G, 1)
    assert ei.value.code == nuri.ERR_LIMIT
    G2 = nuri.load_graph(4, np.array([0, 1], np.int32), np.array([1, 2], np.int32))
    assert nuri.topk_cliques(G2, 1)[0] == (2, (0, 1))
    # a 200-clique is within the limit
    c = list(range(200))
    e = np.array(list(itertools.combinations(c, 2)), np.int32)
    G3 = nuri.load_graph(200, e[:, 0].copy(), e[:, 1].copy())
    r = nuri.topk_cliques(G3, 3)
    assert [x[0] for x in r] == [200, 199, 199]
    assert r[0][1] == tuple(c) and r[1][1] == tuple(c[:199])


def test_device_input_tensors():
    torch = pytest.importorskip("torch")
    g = synth.rmat(10, 8, seed=9)
    s = torch.from_numpy(g.src).cuda()
    d = torch.from_numpy(g.dst).cuda()
    G = nuri.load_graph(g.n, s, d)
    assert [(r[0], r[1]) for r in nuri.topk_cliques(G, 10)] == rows_oracle(g, 10)


def test_chung_lu_scaled_vs_oracle():
    """The headline recipe at n = 20000 (5 planted cliques of 8..12): exact parity with the
    Bron-Kerbosch oracle, both modes (the hub core of this smaller graph holds an 18-clique)."""
    g = synth.chung_lu_planted(20000, 20.0, 2.1, 5, 8, 12, seed=3)
    G = load(g)
    for maximal in (False, True):
        want = [(r[0], tuple(r[1])) for r in oracle.bk_cliques(g, 100, maximal)]
        got = [(r[0], r[1]) for r in nuri.topk_cliques(G, 100, maximal=maximal)]
        assert got == want


def test_chung_lu_config_properties(monkeypatch):
    """Chung-Lu n=1M + 50 planted cliques of 15..30, top-100 (the headline workload).

    The hub block of this graph (the ~600 vertices of expected degree near the cut-off) is
    dense enough to hold background cliques as large as the biggest planted ones, and no CPU
    oracle finishes it in test time; the exact oracle runs on the same recipe at n = 20000
    (test_chung_lu_scaled_vs_oracle).  Here the result is checked through properties that hold
    at any size: every row is a clique of the graph (host adjacency), rows are distinct and in
    rank order, every planted clique above the 100th size is present with all its subsets
    above that size, and a different split of the work (task granularity) gives the same list.
    """
    g = synth.workload("chunglu1m")
    G = load(g)
    got = [(r[0], r[1]) for r in nuri.topk_cliques(G, 100)]
    assert len(got) == 100 and len(set(got)) == 100
    assert got == sorted(got, key=lambda r: (-r[0], r[1]))
    adj = {}
    for a, b in zip(g.src.tolist(), g.dst.tolist()):
        adj.setdefault(a, set()).add(b)
        adj.setdefault(b, set()).add(a)
    assert all(len(r[1]) == r[0] for r in got)
    assert all(all(y in adj[x] for x, y in itertools.combinations(r[1], 2)) for r in got)
    tau = got[-1][0]
    rows = set(r[1] for r in got)
    for c in g.planted:
        c = sorted(c)
        for s in range(len(c), tau, -1):
            for sub in itertools.combinations(c, s):
                assert tuple(sub) in rows
    monkeypatch.setenv("NURI_TASK_SPLIT", "24")
    again = [(r[0], r[1]) for r in nuri.topk_cliques(G, 100)]
    monkeypatch.delenv("NURI_TASK_SPLIT")
    assert again == got
    # a small result set is compacted many times, also between the 4-word and 8-word tiers of
    # one round (the set is replaced while the round is running): same list
    monkeypatch.setenv("NURI_RESULT_CAP", "256")
    small = nuri.topk_cliques(G, 100)
    monkeypatch.delenv("NURI_RESULT_CAP")
    assert [(r[0], r[1]) for r in small] == got


def _near_clique(n, core, missing, p_bg, seed):
    """A clique on `core` random vertices minus `missing` disjoint pairs (2^missing tied
    maximum cliques), plus G(n, p_bg) background edges; ids randomly placed."""
    rng = np.random.default_rng(seed)
    members = rng.choice(n, core, replace=False)
    gone = {tuple(sorted(x)) for x in members[:2 * missing].reshape(missing, 2).tolist()}
    pairs = [(int(a), int(b)) for a, b in itertools.combinations(sorted(members.tolist()), 2)
             if (a, b) not in gone]
    bg = synth.er_small(n, p_bg, seed=seed + 1)
    src = np.concatenate([np.array([a for a, _ in pairs], np.int32), bg.src])
    dst = np.concatenate([np.array([b for _, b in pairs], np.int32), bg.dst])
    return synth.Graph(n, src, dst, name=f"nearclique{core}m{missing}s{seed}")


@pytest.mark.parametrize("core,missing", [(100, 10), (266, 12)])
def test_tie_bound_on_tied_maximum_cliques(monkeypatch, core, missing):
    """Many tied maximum cliques (2^missing of size core - missing): the k rows are the k
    lexicographically smallest, which strict pruning alone finds only by enumerating every
    tie.  The tie bound (a node whose smallest possible sorted id list ranks after the k-th
    known tied result is dropped) must prune and must not change a row: equal to the
    Bron-Kerbosch oracle and to the search with the bound switched off."""
    g = _near_clique(core + 60, core, missing, 0.05, seed=core)
    G = load(g)
    ref = [(r[0], tuple(r[1])) for r in oracle.bk_cliques(g, 300, False)]
    assert ref[0][0] == ref[-1][0] >= core - missing  # at least 300 tied maximum cliques
    pruned = 0
    for k in (1, 5, 50, 300):
        got = nuri.topk_cliques(G, k)
        assert [(r[0], r[1]) for r in got] == ref[:k], k
        pruned += got.stats["lex_pruned"]
    assert pruned > 0
    monkeypatch.setenv("NURI_NO_LEX", "1")
    off = nuri.topk_cliques(G, 50)
    monkeypatch.delenv("NURI_NO_LEX")
    assert [(r[0], r[1]) for r in off] == ref[:50]
    assert off.stats["lex_pruned"] == 0
