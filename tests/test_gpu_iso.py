"""Parity of the CUDA isomorphism path (and hop index) with the oracle; calls go through the
C ABI.  Integer scores and vertex/edge sets: results must match bit-exactly."""
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


def load(g, hops=4):
    return nuri.load_graph(g.n, g.src, g.dst, labels=g.labels, weights=g.weights,
                           index_hops=hops)


def orows(g, q, k, deg=False):
    return [(r[0], tuple(r[1]), tuple(r[2])) for r in oracle.topk_iso(g, q, k, deg)]


def grows(res):
    return [(r[0], r[1], r[2]) for r in res]


def test_fig1b_four_matches():
    d = json.load(open(os.path.join(GOLD, "fig1b_patterns.json")))
    e = np.asarray(d["edges"], np.int32)
    deg = np.bincount(e.ravel(), minlength=d["n"]).astype(np.int32)
    g = synth.Graph(d["n"], e[:, 0].copy(), e[:, 1].copy(),
                    labels=np.asarray(d["labels"], np.uint8), weights=deg)
    G = load(g)
    q = synth.Query(3, d["iso_query"]["labels"], [tuple(x) for x in d["iso_query"]["edges"]])
    for degm in (False, True):
        got = nuri.topk_iso(G, q, 100, degree_rank=degm)
        assert sorted(list(r[1]) for r in got) == sorted(d["iso_matches_vertex_sets"])
        assert grows(got) == orows(g, q, 100, degm)


def _labelled(n, p, seed, nlab=3, wmax=20):
    rng = np.random.default_rng(seed)
    g = synth.er_small(n, p, seed=seed)
    g.labels = rng.integers(0, nlab, size=n).astype(np.uint8)
    g.weights = rng.integers(0, wmax + 1, size=n).astype(np.int32)
    return g


def _shapes(rng, nlab, sizes=(1, 2, 3, 4, 5)):
    out = []
    for kind in ("path", "cycle", "star", "tree"):
        for s in sizes:
            if kind == "cycle" and s < 3:
                continue
            out.append(synth.random_query(rng, kind, s, nlab))
    return out


def test_tiny_vs_oracle_and_brute():
    rng = np.random.default_rng(3)
    for i in range(40):
        g = _labelled(int(rng.integers(2, 12)), [0.3, 0.5, 0.8][i % 3], 700 + i)
        G = load(g, hops=int(rng.integers(0, 4)))
        for q in _shapes(rng, 3):
            for k in (1, 5, 100):
                for degm in (False, True):
                    want = orows(g, q, k, degm)
                    got = grows(nuri.topk_iso(G, q, k, degree_rank=degm))
                    assert got == want, (i, q, k, degm)
                    if i % 8 == 0 and k == 100:
                        assert got == [tuple(r) for r in brute.topk_iso(g, q, k, degm)]


def test_hop_index_vs_oracle():
    for i, g in enumerate([_labelled(300, 0.02, 11, nlab=5, wmax=1000),
                           synth.rmat(11, 8, seed=12)]):
        if g.labels is None:
            rng = np.random.default_rng(5)
            g.labels = rng.integers(0, 8, size=g.n).astype(np.uint8)
            g.weights = rng.integers(0, 1001, size=g.n).astype(np.int32)
        G = load(g, hops=4)
        L = int(g.labels.max()) + 1
        got = nuri.hop_index(G, 4)
        want = oracle.hop_index(g, L, 4, method=1)
        assert np.array_equal(got, want)
        # degree-scored index
        gd = synth.Graph(g.n, g.src, g.dst, labels=g.labels,
                         weights=np.zeros(g.n, np.int32))
        e = {(min(a, b), max(a, b)) for a, b in zip(g.src.tolist(), g.dst.tolist()) if a != b}
        deg = np.zeros(g.n, np.int32)
        for a, b in e:
            deg[a] += 1
            deg[b] += 1
        gd.weights = deg
        assert np.array_equal(nuri.hop_index(G, 4, degree_rank=True),
                              oracle.hop_index(gd, L, 4, method=1))


def test_hop_index_heavy_rows():
    # a hub of degree 3000 exercises the one-CTA-per-vertex kernel
    n = 3100
    src = np.zeros(3000, np.int32)
    dst = np.arange(1, 3001, dtype=np.int32)
    extra = np.arange(3001, 3100, dtype=np.int32)
    src = np.concatenate([src, extra - 1])
    dst = np.concatenate([dst, extra])
    rng = np.random.default_rng(8)
    g = synth.Graph(n, src, dst, labels=rng.integers(0, 8, size=n).astype(np.uint8),
                    weights=rng.integers(0, 1001, size=n).astype(np.int32))
    G = load(g, hops=3)
    assert np.array_equal(nuri.hop_index(G, 3), oracle.hop_index(g, 8, 3, method=1))


def _rmat_labelled(scale, ef, seed, nlab=8):
    g = synth.rmat(scale, ef, seed=seed)
    g.labels = synth.labels_uniform(g.n, nlab, seed=seed + 100)
    g.weights = synth.weights_uniform(g.n, 0, 1000, seed=seed + 200)
    return g


@pytest.mark.parametrize("scale", [10, 12])
def test_rmat_queries_vs_oracle(scale):
    g = _rmat_labelled(scale, 16, seed=scale)
    G = load(g)
    qs = synth.query_batch(12, seed=scale, size_lo=3, size_hi=6, num_labels=8)
    for q in qs:
        for k in (1, 10, 100):
            assert grows(nuri.topk_iso(G, q, k)) == orows(g, q, k), (q, k)


def test_batch_equals_alone():
    g = _rmat_labelled(11, 16, seed=21)
    G = load(g)
    qs = synth.query_batch(16, seed=4, size_lo=3, size_hi=6, num_labels=8)
    ks = [1, 10, 100, 50] * 4
    batch = nuri.topk_iso_batch(G, qs, ks)
    for q, k, b in zip(qs, ks, batch):
        assert grows(b) == grows(nuri.topk_iso(G, q, k))
        assert grows(b) == orows(g, q, k)


def test_special_cases():
    g = _rmat_labelled(10, 8, seed=31, nlab=4)
    G = load(g)
    # 1-vertex query = sort of the label class by weight
    q = synth.Query(1, [2], [])
    v = np.flatnonzero(g.labels == 2)
    order = sorted(v.tolist(), key=lambda x: (-int(g.weights[x]), x))[:30]
    assert grows(nuri.topk_iso(G, q, 30)) == [(int(g.weights[x]), (x,), ()) for x in order]
    # label absent from the graph: no match, no error
    assert list(nuri.topk_iso(G, synth.Query(2, [1, 9], [(0, 1)]), 5)) == []
    # a disconnected query is rejected
    with pytest.raises(nuri.NuriError):
        nuri.topk_iso(G, synth.Query(3, [0, 1, 2], [(0, 1)]), 5)
    with pytest.raises(nuri.NuriError):
        nuri.topk_iso(G, synth.Query(9, [0] * 9, [(i, i + 1) for i in range(8)]), 5)


def test_keep_ties_and_restart(monkeypatch):
    g = _labelled(60, 0.2, 41, nlab=2, wmax=3)   # many equal scores
    G = load(g)
    q = synth.path_query([0, 1, 0])
    allr = brute.topk_iso(g, q, 10 ** 9)
    for k in (1, 7, 40):
        tau = allr[k - 1][0]
        want = [tuple(r) for r in allr if r[0] >= tau]
        assert grows(nuri.topk_iso(G, q, k, keep_ties=True)) == want
    monkeypatch.setenv("NURI_RESULT_CAP", "8")
    got = nuri.topk_iso(G, q, 40)
    monkeypatch.delenv("NURI_RESULT_CAP")
    assert got.stats["restarts"] >= 1
    assert grows(got) == [tuple(r) for r in allr[:40]]


@pytest.mark.parametrize("scale", [10, 12])
def test_rmat_seven_and_eight_vertex_queries_k1000(scale):
    """The largest query sizes of the workloads (7 and 8 vertices, every shape) with
    k = 1000, in one batched launch and one at a time, against the oracle."""
    g = _rmat_labelled(scale, 16, seed=40 + scale)
    G = load(g)
    rng = np.random.default_rng(scale)
    qs = [synth.random_query(rng, kind, s, 8)
          for kind in ("path", "cycle", "star", "tree") for s in (7, 8)]
    batch = nuri.topk_iso_batch(G, qs, [1000] * len(qs))
    for q, b in zip(qs, batch):
        want = orows(g, q, 1000)
        assert grows(b) == want, q
        assert grows(nuri.topk_iso(G, q, 1000)) == want, q


def test_induced_matches_vs_oracle_and_brute():
    """NURI_ISO_INDUCED: only matches whose images of non-adjacent query vertices are
    non-adjacent; compared with the oracle's induced mode (pinned by brute force) on tiny
    graphs and on R-MAT 10 / 12 with k up to 1000."""
    rng = np.random.default_rng(5)
    for i in range(20):
        g = _labelled(int(rng.integers(3, 12)), [0.4, 0.7][i % 2], 1700 + i, nlab=2)
        G = load(g)
        for q in _shapes(rng, 2, sizes=(2, 3, 4, 5)):
            for k in (1, 100):
                want = [(r[0], tuple(r[1]), tuple(r[2])) for r in oracle.topk_iso(g, q, k, induced=True)]
                assert grows(nuri.topk_iso(G, q, k, induced=True)) == want, (i, q, k)
                if i % 5 == 0:
                    assert want == [tuple(r) for r in brute.topk_iso(g, q, k, induced=True)]
    for scale in (10, 12):
        g = _rmat_labelled(scale, 16, seed=60 + scale, nlab=4)
        G = load(g)
        qs = synth.query_batch(12, seed=scale + 3, size_lo=3, size_hi=7, num_labels=4)
        got = nuri.topk_iso_batch(G, qs, [1000] * len(qs), induced=True)
        for q, r in zip(qs, got):
            want = [(x[0], tuple(x[1]), tuple(x[2])) for x in oracle.topk_iso(g, q, 1000, induced=True)]
            assert grows(r) == want, q


def test_matched_vertex_bound_same_rows_fewer_candidates(monkeypatch):
    """The bound of an unmatched query vertex taken from the nearest matched image (not only
    the root's) prunes more and changes no row: equal to the root-only bound and the oracle."""
    g = _rmat_labelled(12, 16, seed=71)
    G = load(g)
    qs = synth.query_batch(16, seed=72, size_lo=5, size_hi=8, num_labels=8)
    tight = nuri.topk_iso_batch(G, qs, [100] * len(qs))
    monkeypatch.setenv("NURI_ISO_ROOT_BOUND", "1")
    loose = nuri.topk_iso_batch(G, qs, [100] * len(qs))
    monkeypatch.delenv("NURI_ISO_ROOT_BOUND")
    for q, a, b in zip(qs, tight, loose):
        assert grows(a) == grows(b) == orows(g, q, 100), q
    assert tight[0].stats["expansions"] <= loose[0].stats["expansions"]


def _edge_weighted(g, seed, hi=100, dup=True):
    """One weight per input pair (uniform 0..hi); with dup, a third of the pairs come once
    more, reversed, with their own weight (an edge weighs the larger)."""
    rng = np.random.default_rng(seed)
    if dup and g.m:
        pick = rng.integers(0, g.m, size=max(1, g.m // 3))
        g.src, g.dst = (np.concatenate([g.src, g.dst[pick]]).astype(np.int32),
                        np.concatenate([g.dst, g.src[pick]]).astype(np.int32))
    g.edge_weights = rng.integers(0, hi + 1, size=g.m).astype(np.int32)
    return g


def load_ew(g, hops=2):
    G = load(g, hops)
    G.set_edge_weights(g.src, g.dst, g.edge_weights)
    return G


def orows_e(g, q, k, induced=False):
    return [(r[0], tuple(r[1]), tuple(r[2]))
            for r in oracle.topk_iso(g, q, k, induced=induced, edge_rank=True)]


def test_edge_rank_tiny_vs_oracle_and_brute():
    """Ranking by cumulative edge weight (NURI_RANK_EDGE_WEIGHT_SUM) on tiny labelled graphs:
    the CUDA rows equal the oracle's and brute force's, non-induced and induced."""
    rng = np.random.default_rng(17)
    for i in range(30):
        g = _edge_weighted(_labelled(int(rng.integers(2, 12)), [0.3, 0.5, 0.8][i % 3], 1700 + i),
                           seed=i, hi=[3, 40][i % 2])
        G = load_ew(g, hops=int(rng.integers(0, 3)))
        for q in _shapes(rng, 3, sizes=(1, 2, 3, 4, 6)):
            for induced in (False, True):
                every = [tuple(r) for r in brute.topk_iso(g, q, 10 ** 9, induced=induced,
                                                          edge_rank=True)]
                for k in (1, 5, 100):
                    got = grows(nuri.topk_iso(G, q, k, induced=induced, edge_rank=True))
                    assert got == every[:k], (g.name, q, k, induced)
                    assert orows_e(g, q, k, induced) == every[:k]


@pytest.mark.parametrize("scale", [10, 12])
def test_edge_rank_rmat_vs_oracle(scale):
    """R-MAT 10 / 12 with 8 labels and edge weights 0..1000: queries of 3 to 8 vertices
    (every shape), k up to 1000, one batched launch and one query at a time."""
    g = _edge_weighted(_rmat_labelled(scale, 16, seed=60 + scale), seed=scale, hi=1000)
    G = load_ew(g)
    rng = np.random.default_rng(70 + scale)
    qs = [synth.random_query(rng, kind, s, 8)
          for kind in ("path", "cycle", "star", "tree") for s in (3, 5, 8)]
    ks = [1, 10, 100, 1000] * 3
    batch = nuri.topk_iso_batch(G, qs, ks, edge_rank=True)
    for q, k, b in zip(qs, ks, batch):
        want = orows_e(g, q, k)
        assert grows(b) == want, (q, k)
        assert grows(nuri.topk_iso(G, q, k, edge_rank=True)) == want, (q, k)
    # the same graph still ranks by vertex weight when asked
    q = qs[1]
    assert grows(nuri.topk_iso(G, q, 10)) == orows(g, q, 10)


def test_edge_rank_inputs_and_errors():
    torch = pytest.importorskip("torch")
    g = _edge_weighted(_rmat_labelled(10, 8, seed=81, nlab=4), seed=3, hi=50, dup=False)
    G = load(g)
    q = synth.cycle_query([0, 1, 2])
    with pytest.raises(nuri.NuriError):  # no edge weights yet
        nuri.topk_iso(G, q, 5, edge_rank=True)
    # device tensors give the same weights as host arrays
    G.set_edge_weights(torch.from_numpy(g.src).cuda(), torch.from_numpy(g.dst).cuda(),
                       torch.from_numpy(g.edge_weights).cuda())
    assert grows(nuri.topk_iso(G, q, 50, edge_rank=True)) == orows_e(g, q, 50)
    # a pair that is not an edge, a negative weight, an id out of range: rejected, and the
    # weights set before stay in use
    adj = {(int(a), int(b)) for a, b in zip(g.src, g.dst)} | \
        {(int(b), int(a)) for a, b in zip(g.src, g.dst)}
    non = next((a, b) for a in range(g.n) for b in range(a + 1, g.n) if (a, b) not in adj)
    for s, d, w in ((non[0], non[1], 1), (int(g.src[0]), int(g.dst[0]), -1), (0, g.n, 1)):
        with pytest.raises(nuri.NuriError) as ei:
            G.set_edge_weights(np.array([s], np.int32), np.array([d], np.int32),
                               np.array([w], np.int32))
        assert ei.value.code == nuri.ERR_INVALID
    assert grows(nuri.topk_iso(G, q, 50, edge_rank=True)) == orows_e(g, q, 50)
    # edges given no weight weigh 0: weighting only the first pair
    G.set_edge_weights(g.src[:1], g.dst[:1], np.array([7], np.int32))
    top = nuri.topk_iso(G, synth.path_query([int(g.labels[g.src[0]]), int(g.labels[g.dst[0]])]),
                        1, edge_rank=True)
    if g.src[0] != g.dst[0]:
        assert top[0][0] == 7
    # mixed batch: the same query ranked three ways
    G.set_edge_weights(g.src, g.dst, g.edge_weights)
    outs = nuri.topk_batch(G, [("iso", q, 20), ("iso", q, 20, "edge"), ("iso", q, 20, True)])
    assert grows(outs[1]) == orows_e(g, q, 20)
    assert grows(outs[0]) == orows(g, q, 20)
    assert grows(outs[2]) == orows(g, q, 20, True)
    # an unlabelled graph has no label segments
    U = nuri.load_graph(g.n, g.src, g.dst)
    with pytest.raises(nuri.NuriError):
        U.set_edge_weights(g.src, g.dst, g.edge_weights)


def test_edge_rank_rmat14_batch_vs_oracle():
    """Sixteen seeded queries (3 to 8 vertices) on R-MAT 14 with 8 labels and edge weights
    0..1000, top-100 by cumulative edge weight, in one batched launch: every row equal to the
    oracle's (about 10 s of oracle time)."""
    g = _rmat_labelled(14, 16, seed=14)
    g.edge_weights = synth.edge_weights_uniform(g.m, 0, 1000, seed=314)
    G = load_ew(g)
    qs = synth.query_batch(16, seed=3, size_lo=3, size_hi=8, num_labels=8)
    batch = nuri.topk_iso_batch(G, qs, [100] * len(qs), edge_rank=True)
    for q, b in zip(qs, batch):
        assert grows(b) == orows_e(g, q, 100), q
