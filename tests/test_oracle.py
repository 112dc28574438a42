"""Pins of the oracle against what the paper and the mathematics fix (CPU only).

* the paper's worked examples (tests/golden/*.json, each with its citation);
* brute force from the definitions (oracle/brute.py) on many seeded tiny graphs;
* Bron-Kerbosch, an independent clique algorithm;
* closed forms on planted-clique graphs;
* special cases that reduce to a sort or to triangle listing;
* invariants the paper states (anti-monotone support, hop-index monotonicity).
"""
import itertools
import json
import os

import numpy as np
import pytest

import oracle
import synth
from oracle import brute

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def gold(name):
    with open(os.path.join(GOLD, name)) as f:
        return json.load(f)


def graph_from(d, labels=None, weights=None):
    e = np.asarray(d["edges"], dtype=np.int32)
    return synth.Graph(d["n"], e[:, 0].copy(), e[:, 1].copy(),
                       labels=None if labels is None else np.asarray(labels, np.uint8),
                       weights=None if weights is None else np.asarray(weights, np.int32))


# ------------------------------------------------------------------------------------------
# cliques
# ------------------------------------------------------------------------------------------
def test_fig1a_topk_lists():
    d = gold("fig1a_cliques.json")
    g = graph_from(d)
    for k, expect in d["topk"].items():
        rows = oracle.topk_cliques(g, int(k))
        assert [list(r[1]) for r in rows] == expect
        assert [r[0] for r in rows] == [len(x) for x in expect]
    assert len(oracle.topk_cliques(g, 100)) == d["num_cliques"]
    assert len(brute.all_cliques(g)) == d["num_cliques"]
    rows = oracle.topk_cliques(g, 10, maximal=True)
    assert [list(r[1]) for r in rows] == d["maximal"]


def test_fig1a_trace_counts():
    d = gold("fig1a_cliques.json")
    g = graph_from(d)
    r = oracle.topk_cliques(g, 1)
    assert r.expansions == d["top1_trace"]["children_created"]
    assert r.dequeued == d["top1_trace"]["unit_subgraphs"] + d["top1_trace"]["children_created"]


def _tiny_graphs(count, seed0=100):
    rng = np.random.default_rng(seed0)
    for i in range(count):
        n = int(rng.integers(1, 15))
        p = [0.2, 0.5, 0.8][i % 3]
        yield synth.er_small(n, p, seed=seed0 + i)


def test_cliques_oracle_vs_brute_and_bk():
    for g in _tiny_graphs(240):
        for k in (1, 3, 10, 60):
            for maximal in (False, True):
                want = [(s, tuple(c)) for s, c in brute.topk_cliques(g, k, maximal)]
                got = [(r[0], r[1]) for r in oracle.topk_cliques(g, k, maximal)]
                assert got == want, (g.name, k, maximal)
                bk = [(r[0], r[1]) for r in oracle.bk_cliques(g, k, maximal)]
                assert bk == want, (g.name, k, maximal, "bk")


def test_cliques_nonprune_equivalent_budget_flag():
    # a work budget stops the run early and says so
    g = synth.er_small(30, 0.5, seed=7)
    r = oracle.topk_cliques(g, 5, budget=10)
    assert not r.complete
    r = oracle.topk_cliques(g, 5)
    assert r.complete


def test_cliques_closed_form_planted_er():
    """ER(2000, 0.01) + planted 12-clique C: top-10 = [C, C - c12, C - c11, ..., C - c4]."""
    g = synth.workload("er2000")
    C = sorted(g.planted[0])
    # assumption of the closed form: no other clique reaches size 11
    mx = oracle.bk_cliques(g, 2, True)
    assert list(mx[0][1]) == C and mx[1][0] < 11
    want = [tuple(C)] + [tuple(x for x in C if x != C[j]) for j in range(11, 2, -1)]
    got = [r[1] for r in oracle.topk_cliques(g, 10)]
    assert got == want
    # k = 1 is the textbook maximum clique
    assert oracle.topk_cliques(g, 1)[0][1] == tuple(C)


def test_cliques_closed_form_small_planted():
    """Two disjoint planted cliques of sizes 7 and 6 in a sparse graph: all-cliques ranking."""
    rng = np.random.default_rng(3)
    n = 200
    base = synth.er_small(n, 0.01, seed=5)
    a = sorted(rng.choice(n, 13, replace=False).tolist())
    c7, c6 = a[:7], a[7:]
    extra = [(x, y) for c in (c7, c6) for x, y in itertools.combinations(c, 2)]
    src = np.concatenate([base.src, np.array([e[0] for e in extra], np.int32)])
    dst = np.concatenate([base.dst, np.array([e[1] for e in extra], np.int32)])
    g = synth.Graph(n, src, dst)
    bk = oracle.bk_cliques(g, 3, True)
    assert [list(r[1]) for r in bk[:2]] == [c7, c6] and bk[2][0] <= 4
    # sizes 7 (1 clique), 6 (7 subsets of c7 + c6 itself), 5 (21 + 6) ...
    def subsets(c, s):
        return [tuple(x) for x in itertools.combinations(c, s)]
    want = [tuple(c7)] + sorted(subsets(c7, 6) + [tuple(c6)]) + sorted(subsets(c7, 5) + subsets(c6, 5))
    got = [r[1] for r in oracle.topk_cliques(g, len(want))]
    assert got == want


def test_cliques_closed_form_tied_maxima_matching_complement():
    """A complete graph minus a perfect matching on 2t of its vertices: every maximal clique
    takes the universal vertices and one end of each missing edge, so there are 2^t tied
    maximum cliques.  Ranked by sorted id list, two of them first differ at the missing edge
    with the smallest lower end among those where they choose differently, and the one taking
    that lower end ranks first.  With the missing edges ordered by lower end, the r-th
    maximum clique therefore takes the upper end exactly where the binary digits of r (most
    significant first) are 1.  Algorithm 1 and BK must produce these rows; the search's tie
    handling on near-cliques rests on this order."""
    rng = np.random.default_rng(11)
    n, t = 26, 6
    ids = rng.permutation(n)
    pairs = [tuple(sorted((int(ids[2 * i]), int(ids[2 * i + 1])))) for i in range(t)]
    universal = sorted(int(x) for x in ids[2 * t:])
    missing = set(pairs)
    edges = [(a, b) for a, b in itertools.combinations(range(n), 2) if (a, b) not in missing]
    g = synth.Graph(n, np.array([e[0] for e in edges], np.int32),
                    np.array([e[1] for e in edges], np.int32))
    pairs.sort()  # by lower end
    want = []
    for r in range(2 ** t):
        pick = [pairs[j][(r >> (t - 1 - j)) & 1] for j in range(t)]
        want.append((n - t, tuple(sorted(universal + pick))))
    for k in (1, 5, 17, 64):
        assert [(r[0], r[1]) for r in oracle.topk_cliques(g, k)] == want[:k], k
        assert [(r[0], r[1]) for r in oracle.bk_cliques(g, k, False)] == want[:k], k
    # every maximal clique is one of them: the maximal ranking stops at 2^t rows
    assert [(r[0], r[1]) for r in oracle.bk_cliques(g, 100, True)] == want


# ------------------------------------------------------------------------------------------
# subgraph isomorphism
# ------------------------------------------------------------------------------------------
def test_fig1b_iso_four_matches():
    d = gold("fig1b_patterns.json")
    deg = [0] * d["n"]
    for a, b in d["edges"]:
        deg[a] += 1
        deg[b] += 1
    g = graph_from(d, d["labels"], deg)
    q = synth.Query(3, d["iso_query"]["labels"], [tuple(e) for e in d["iso_query"]["edges"]])
    rows = oracle.topk_iso(g, q, 100)
    assert sorted(list(r[1]) for r in rows) == sorted(d["iso_matches_vertex_sets"])
    # the paper ranks by degree sum; with weights = degrees both modes agree
    rows_d = oracle.topk_iso(g, q, 100, degree_rank=True)
    assert [r[:3] for r in rows_d] == [r[:3] for r in rows]
    # the stated bijection mu(0)=v1, mu(1)=v2, mu(2)=v3 is one of the matches
    assert any(r[1] == (0, 1, 2) and set(r[2]) == {(0, 1), (1, 2)} for r in rows)


def _tiny_labelled(count, seed0=300, nlab=3):
    rng = np.random.default_rng(seed0)
    for i in range(count):
        n = int(rng.integers(2, 10))
        g = synth.er_small(n, [0.3, 0.5, 0.7][i % 3], seed=seed0 + i)
        g.labels = rng.integers(0, nlab, size=n).astype(np.uint8)
        g.weights = rng.integers(0, 20, size=n).astype(np.int32)
        yield g


def _queries(rng, nlab):
    out = []
    for kind, sizes in (("path", (1, 2, 3, 4)), ("cycle", (3, 4)), ("star", (3, 4)),
                        ("tree", (4, 5))):
        for s in sizes:
            out.append(synth.random_query(rng, kind, s, nlab))
    return out


def test_iso_oracle_vs_brute():
    rng = np.random.default_rng(11)
    for g in _tiny_labelled(60):
        for q in _queries(rng, 3):
            for k in (1, 4, 50):
                for deg in (False, True):
                    want = brute.topk_iso(g, q, k, deg)
                    got = [r[:3] for r in oracle.topk_iso(g, q, k, deg)]
                    assert got == want, (g.name, q, k, deg)


def _clean_edges(g):
    e = {(min(a, b), max(a, b)) for a, b in zip(g.src.tolist(), g.dst.tolist()) if a != b}
    return sorted(e)


def test_iso_special_case_single_vertex_is_a_sort():
    g = synth.rmat(9, 8, seed=4)
    rng = np.random.default_rng(2)
    g.labels = rng.integers(0, 4, size=g.n).astype(np.uint8)
    g.weights = rng.integers(0, 1001, size=g.n).astype(np.int32)
    q = synth.Query(1, [2], [])
    got = [(r[0], r[1]) for r in oracle.topk_iso(g, q, 25)]
    v = np.flatnonzero(g.labels == 2)
    order = sorted(v.tolist(), key=lambda x: (-int(g.weights[x]), x))[:25]
    assert got == [(int(g.weights[x]), (x,)) for x in order]


def test_iso_special_case_edge_query_is_an_edge_sort():
    g = synth.rmat(9, 8, seed=5)
    rng = np.random.default_rng(3)
    g.labels = rng.integers(0, 3, size=g.n).astype(np.uint8)
    g.weights = rng.integers(0, 1001, size=g.n).astype(np.int32)
    for la, lb in ((0, 1), (2, 2)):
        q = synth.Query(2, [la, lb], [(0, 1)])
        rows = []
        for a, b in _clean_edges(g):
            if {int(g.labels[a]), int(g.labels[b])} == {la, lb} and \
               sorted([int(g.labels[a]), int(g.labels[b])]) == sorted([la, lb]):
                rows.append((int(g.weights[a]) + int(g.weights[b]), (a, b), ((a, b),)))
        rows.sort(key=lambda r: (-r[0], r[1], r[2]))
        got = [r[:3] for r in oracle.topk_iso(g, q, 40)]
        assert got == rows[:40]


def test_iso_special_case_triangle_listing():
    g = synth.rmat(8, 8, seed=6)
    rng = np.random.default_rng(4)
    g.labels = rng.integers(0, 2, size=g.n).astype(np.uint8)
    g.weights = rng.integers(0, 100, size=g.n).astype(np.int32)
    A = np.zeros((g.n, g.n), dtype=bool)
    for a, b in _clean_edges(g):
        A[a, b] = A[b, a] = True
    tri = []
    for a in range(g.n):
        for b in np.flatnonzero(A[a, a + 1:]) + a + 1:
            for c in np.flatnonzero(A[a, b + 1:] & A[b, b + 1:]) + b + 1:
                tri.append((a, int(b), int(c)))
    q = synth.cycle_query([0, 0, 1])
    want = []
    for t in tri:
        if sorted(int(g.labels[x]) for x in t) == [0, 0, 1]:
            want.append((int(sum(g.weights[x] for x in t)), t,
                         tuple(sorted(itertools.combinations(t, 2)))))
    want.sort(key=lambda r: (-r[0], r[1], r[2]))
    got = [r[:3] for r in oracle.topk_iso(g, q, 10 ** 6)]
    assert got == want


def test_hop_index_walk_definition_vs_recurrence():
    rng = np.random.default_rng(9)
    for i in range(25):
        g = synth.er_small(int(rng.integers(2, 25)), 0.15, seed=900 + i)
        g.labels = rng.integers(0, 3, size=g.n).astype(np.uint8)
        g.weights = rng.integers(0, 50, size=g.n).astype(np.int32)
        a = oracle.hop_index(g, 3, 4, method=0)
        b = oracle.hop_index(g, 3, 4, method=1)
        assert np.array_equal(a, b)
        # cumulative hops: non-decreasing in h
        assert np.all(np.diff(a, axis=0) >= 0)


def test_hop_index_hand_worked_path():
    # path 0-1-2-3, labels (0,1,0,1), weights (5,7,9,3)
    g = synth.Graph(4, np.array([0, 1, 2], np.int32), np.array([1, 2, 3], np.int32),
                    labels=np.array([0, 1, 0, 1], np.uint8),
                    weights=np.array([5, 7, 9, 3], np.int32))
    idx = oracle.hop_index(g, 2, 3, method=0)
    # h=1: neighbours only
    assert idx[0].tolist() == [[-1, 7], [9, -1], [-1, 7], [9, -1]]
    # h=2: walks of length 1..2 (a vertex reaches itself through a neighbour)
    assert idx[1].tolist() == [[9, 7], [9, 7], [9, 7], [9, 7]]
    # h=3 from vertex 0 reaches vertex 3 (weight 3 < 7): unchanged
    assert idx[2][0].tolist() == [9, 7]


# ------------------------------------------------------------------------------------------
# patterns
# ------------------------------------------------------------------------------------------
def test_fig1b_supports_and_top_pattern():
    d = gold("fig1b_patterns.json")
    g = graph_from(d, d["labels"])
    for p in d["patterns"]:
        f, dom = oracle.mni(g, p["labels"], p["edges"])
        assert f == p["f"] and dom == p["domains"], p["name"]
        bf, bdom = brute.pattern_mni(g, len(p["labels"]), p["labels"], [tuple(e) for e in p["edges"]])
        assert bf == p["f"] and bdom == p["domains"]
    top = oracle.topk_patterns(g, 2, 1)
    assert top[0][0] == d["top1_2edge"]["f"] and list(top[0][3]) == d["top1_2edge"]["labels"]
    # 1-edge groups: a-b (2 directed minimal codes) and b-b (6)
    one = oracle.topk_patterns(g, 1, 10)
    assert sorted((r[0], r[3]) for r in one) == [(2, (0, 1)), (3, (1, 1))]


def _tiny_pattern_graphs(count, seed0=500):
    rng = np.random.default_rng(seed0)
    for i in range(count):
        n = int(rng.integers(3, 9))
        g = synth.er_small(n, [0.3, 0.5][i % 2], seed=seed0 + i)
        g.labels = rng.integers(0, 2 + i % 2, size=n).astype(np.uint8)
        yield g


def test_patterns_oracle_vs_brute():
    for g in _tiny_pattern_graphs(40):
        for M in (1, 2, 3):
            for k in (1, 3, 20):
                want = brute.topk_patterns(g, M, k)
                got = oracle.topk_patterns(g, M, k)
                got2 = [(r[0], brute.code_from_row(len(r[1]), r[3], r[2])) for r in got]
                assert got2 == want, (g.name, M, k)


def test_patterns_m1_closed_form():
    """f(l1-l2) = min(#l1 vertices with an l2 neighbour, #l2 vertices with an l1 neighbour)."""
    g = synth.rmat(10, 8, seed=8)
    g.labels = synth.labels_zipf(g.n, 5, 1.2, seed=8)
    E = np.array(_clean_edges(g), dtype=np.int64)
    L = g.labels.astype(np.int64)
    la, lb = L[E[:, 0]], L[E[:, 1]]
    expect = {}
    for x in range(5):
        for y in range(x, 5):
            m1 = ((la == x) & (lb == y))
            m2 = ((la == y) & (lb == x))
            if not (m1.any() or m2.any()):
                continue
            side_x = set(E[m1, 0].tolist()) | set(E[m2, 1].tolist())
            side_y = set(E[m1, 1].tolist()) | set(E[m2, 0].tolist())
            expect[(x, y)] = len(side_x | side_y) if x == y else min(len(side_x), len(side_y))
    rows = oracle.topk_patterns(g, 1, 100)
    got = {tuple(sorted(r[3])): r[0] for r in rows}
    assert got == expect


def test_patterns_anti_monotone():
    g = synth.rmat(9, 8, seed=12)
    g.labels = synth.labels_zipf(g.n, 3, 1.2, seed=12)
    rng = np.random.default_rng(5)
    for _ in range(12):
        # random connected pattern with 3 vertices and its 1-edge sub-patterns
        labs = rng.integers(0, 3, size=3).tolist()
        f3, _ = oracle.mni(g, labs, [(0, 1), (1, 2)])
        fa, _ = oracle.mni(g, labs[:2], [(0, 1)])
        fb, _ = oracle.mni(g, labs[1:], [(0, 1)])
        assert f3 <= fa and f3 <= fb
        ft, _ = oracle.mni(g, labs, [(0, 1), (1, 2), (0, 2)])
        assert ft <= f3


def test_canonical_code_invariant_under_relabelling():
    rng = np.random.default_rng(6)
    for _ in range(30):
        nv = int(rng.integers(2, 6))
        labs = rng.integers(0, 3, size=nv).tolist()
        edges = [(i, int(rng.integers(0, i))) for i in range(1, nv)]
        code, _ = oracle.canonical_code(labs, edges)
        perm = rng.permutation(nv).tolist()
        labs2 = [0] * nv
        for i in range(nv):
            labs2[perm[i]] = labs[i]
        edges2 = [(perm[a], perm[b]) for a, b in edges]
        code2, _ = oracle.canonical_code(labs2, edges2)
        assert code == code2 == brute.canon_code(nv, labs, edges)


def test_iso_oracle_vs_brute_six_to_eight_vertex_queries():
    """Algorithm 1 with the isomorphism functions, pinned by brute force at the query sizes
    of the R-MAT workloads (6, 7 and 8 vertices, every shape), both score modes."""
    rng = np.random.default_rng(29)
    for i in range(8):
        n = int(rng.integers(8, 12))
        g = synth.er_small(n, [0.45, 0.6][i % 2], seed=900 + i)
        g.labels = rng.integers(0, 2, size=n).astype(np.uint8)
        g.weights = rng.integers(0, 30, size=n).astype(np.int32)
        for kind in ("path", "cycle", "star", "tree"):
            for s in (6, 7, 8):
                q = synth.random_query(rng, kind, s, 2)
                for k in (1, 10, 1000):
                    for deg in (False, True):
                        want = brute.topk_iso(g, q, k, deg)
                        got = [r[:3] for r in oracle.topk_iso(g, q, k, deg)]
                        assert got == want, (g.name, q, k, deg)


def test_patterns_oracle_vs_brute_four_and_five_edges():
    """Algorithm 2 with MNI support, pinned by brute force at M = 4 and M = 5 (patterns of up
    to 6 vertices, the sizes of the R-MAT 18 workload) on 7-vertex graphs."""
    rng = np.random.default_rng(31)
    for i in range(6):
        g = synth.er_small(7, [0.45, 0.6][i % 2], seed=950 + i)
        g.labels = rng.integers(0, 2 + i % 2, size=7).astype(np.uint8)
        for M in (4, 5):
            for k in (1, 5, 50):
                want = brute.topk_patterns(g, M, k)
                got = oracle.topk_patterns(g, M, k)
                got2 = [(r[0], brute.code_from_row(len(r[1]), r[3], r[2])) for r in got]
                assert got2 == want, (g.name, M, k)


def test_iso_oracle_induced_vs_brute():
    """The induced reading (non-adjacent query vertices map to non-adjacent data vertices),
    pinned by brute force; every induced match is also a non-induced one."""
    rng = np.random.default_rng(37)
    for g in _tiny_labelled(40, seed0=1300, nlab=2):
        for q in _queries(rng, 2):
            for k in (1, 5, 100):
                for deg in (False, True):
                    want = brute.topk_iso(g, q, k, deg, induced=True)
                    got = [r[:3] for r in oracle.topk_iso(g, q, k, deg, induced=True)]
                    assert got == want, (g.name, q, k, deg)
                    every = {r[1:3] for r in brute.topk_iso(g, q, 10 ** 9, deg)}
                    assert all(r[1:3] in every for r in got)
    # a path a-b-c inside a triangle is a non-induced match but not an induced one
    g = synth.Graph(3, np.array([0, 1, 0], np.int32), np.array([1, 2, 2], np.int32),
                    labels=np.zeros(3, np.uint8), weights=np.ones(3, np.int32))
    q = synth.path_query([0, 0, 0])
    assert len(oracle.topk_iso(g, q, 10)) == 3
    assert len(oracle.topk_iso(g, q, 10, induced=True)) == 0


def _with_edge_weights(g, rng, hi=25):
    """One weight per input pair; a third of the pairs are given once more, reversed, with
    a weight of their own (an edge then weighs the larger of the two)."""
    if g.m:
        pick = rng.integers(0, g.m, size=max(1, g.m // 3))
        src = np.concatenate([g.src, g.dst[pick]]).astype(np.int32)
        dst = np.concatenate([g.dst, g.src[pick]]).astype(np.int32)
        g.src, g.dst = src, dst
    g.edge_weights = rng.integers(0, hi + 1, size=g.m).astype(np.int32)
    return g


def test_iso_oracle_edge_rank_vs_brute():
    """Ranking by cumulative edge weight (Section 2, top-k semantics: the matches of the
    highest cumulative edge weight), pinned by brute force: every image scored by the sum of
    its edges' weights, non-induced and induced, queries of 1 to 6 vertices."""
    rng = np.random.default_rng(41)
    for g in _tiny_labelled(50, seed0=1500, nlab=2):
        g = _with_edge_weights(g, rng)
        qs = _queries(rng, 2) + [synth.random_query(rng, "tree", 6, 2)]
        for q in qs:
            for k in (1, 4, 50):
                for induced in (False, True):
                    want = brute.topk_iso(g, q, k, induced=induced, edge_rank=True)
                    got = [r[:3] for r in oracle.topk_iso(g, q, k, induced=induced,
                                                          edge_rank=True)]
                    assert got == want, (g.name, q, k, induced)


def test_iso_oracle_edge_rank_worked_example():
    """Two disjoint triangles: {0,1,2} with edge weights 1, 1, 1 and {3,4,5} with 5, 1, 1.
    The heavier triangle wins (7 > 3) until the pair (1, 0) is given again with weight 9: an
    edge weighs the largest weight given for it, so {0,1,2} then weighs 11."""
    src = np.array([0, 1, 2, 3, 4, 5], np.int32)
    dst = np.array([1, 2, 0, 4, 5, 3], np.int32)
    w = np.array([1, 1, 1, 5, 1, 1], np.int32)
    g = synth.Graph(6, src, dst, labels=np.zeros(6, np.uint8), weights=np.ones(6, np.int32),
                    edge_weights=w)
    tri = synth.cycle_query([0, 0, 0])
    edge = synth.path_query([0, 0])
    assert [r[:2] for r in oracle.topk_iso(g, tri, 2, edge_rank=True)] == [
        (7, (3, 4, 5)), (3, (0, 1, 2))]
    assert [r[:2] for r in oracle.topk_iso(g, edge, 3, edge_rank=True)] == [
        (5, (3, 4)), (1, (0, 1)), (1, (0, 2))]
    g2 = synth.Graph(6, np.append(src, 1).astype(np.int32), np.append(dst, 0).astype(np.int32),
                     labels=g.labels, weights=g.weights,
                     edge_weights=np.append(w, 9).astype(np.int32))
    assert [r[:2] for r in oracle.topk_iso(g2, tri, 2, edge_rank=True)] == [
        (11, (0, 1, 2)), (7, (3, 4, 5))]
    assert oracle.topk_iso(g2, edge, 1, edge_rank=True)[0][:2] == (9, (0, 1))


def test_weighted_cliques_oracle_vs_brute():
    """Cliques ranked by the sum of vertex weights (Algorithm 1 with the weighted bound
    w(V) + w(P)), pinned by brute force on tiny graphs: all cliques and maximal ones."""
    rng = np.random.default_rng(43)
    for i in range(60):
        n = int(rng.integers(1, 11))
        g = synth.er_small(n, [0.3, 0.5, 0.8][i % 3], seed=1600 + i)
        g.weights = rng.integers(0, [3, 50][i % 2] + 1, size=n).astype(np.int32)
        for k in (1, 3, 10, 1000):
            for maximal in (False, True):
                want = [(s, tuple(c)) for s, c in brute.topk_wcliques(g, k, maximal)]
                got = [(r[0], tuple(r[1])) for r in oracle.topk_wcliques(g, k, maximal)]
                assert got == want, (g.name, k, maximal)


def test_weighted_cliques_unit_weights_rank_by_size():
    """With every weight 1 the weighted ranking is the ranking by size (Algorithm 1 with the
    unweighted functions), on graphs beyond brute force."""
    for seed in (3, 4):
        g = synth.rmat(9, 8, seed=seed)
        g.weights = np.ones(g.n, np.int32)
        for k in (1, 30, 300):
            want = [(r[0], tuple(r[1])) for r in oracle.topk_cliques(g, k)]
            assert [(r[0], tuple(r[1])) for r in oracle.topk_wcliques(g, k)] == want
