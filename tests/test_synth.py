"""The seeded input generators follow their stated recipes (CPU): the shapes and
distributions the workloads are meant to have, and determinism under a fixed seed."""
import itertools

import numpy as np

import synth


def _edge_set(g):
    keep = g.src != g.dst
    a = np.minimum(g.src[keep], g.dst[keep]).astype(np.int64)
    b = np.maximum(g.src[keep], g.dst[keep]).astype(np.int64)
    return set((a * g.n + b).tolist())


def test_er2000_density_and_planted_clique():
    g = synth.workload("er2000")
    e = _edge_set(g)
    # G(2000, 0.01): about 0.01 * C(2000, 2) = 19990 pairs, plus at most 66 planted ones
    assert abs(len(e) - 19990) < 600
    assert len(g.planted) == 1 and len(g.planted[0]) == 12
    for u, v in itertools.combinations(sorted(g.planted[0]), 2):
        assert u * g.n + v in e


def test_chung_lu_small_mean_degree_and_disjoint_planted_cliques():
    g = synth.chung_lu_planted(20000, 20.0, 2.1, 10, 8, 16, seed=7)
    e = _edge_set(g)
    mean_deg = 2 * len(e) / g.n
    assert 15.0 < mean_deg < 21.0  # duplicates and self-loops of the 10 n draws removed
    seen = set()
    for c in g.planted:
        assert 8 <= len(c) <= 16
        assert not (set(c) & seen)
        seen |= set(c)
        for u, v in itertools.combinations(sorted(c), 2):
            assert u * g.n + v in e


def test_zipf_labels_follow_their_law():
    lab = synth.labels_zipf(200000, 16, 1.2, seed=3)
    p = np.arange(1, 17, dtype=np.float64) ** -1.2
    p /= p.sum()
    freq = np.bincount(lab, minlength=16) / lab.size
    assert abs(freq[0] - p[0]) < 0.01  # label 0 about 36.5 %
    assert np.all(np.diff(freq) < 0.01)  # non-increasing up to noise


def test_rmat_labels_weights_and_determinism():
    g1 = synth.workload("rmat18z")
    g2 = synth.workload("rmat18z")
    assert g1.n == 1 << 18 and g1.src.size == 16 << 18
    assert np.array_equal(g1.src, g2.src) and np.array_equal(g1.labels, g2.labels)
    assert g1.labels.max() < 16
    w = synth.weights_uniform(10000, 0, 1000, seed=11)
    assert w.min() >= 0 and w.max() <= 1000 and w.dtype == np.int32


def test_query_batch_shapes():
    qs = synth.query_batch(64, seed=1)
    assert len(qs) == 64
    for q in qs:
        assert 4 <= q.nq <= 8 and len(q.labels) == q.nq
        # connected: every vertex reachable from vertex 0
        adj = {i: set() for i in range(q.nq)}
        for a, b in q.edges:
            adj[a].add(b)
            adj[b].add(a)
        seen, todo = {0}, [0]
        while todo:
            x = todo.pop()
            for y in adj[x] - seen:
                seen.add(y)
                todo.append(y)
        assert len(seen) == q.nq


def test_chung_lu_expected_degrees_clipped_with_mean_kept():
    # the stated recipe: mean expected degree 20, every weight at most sqrt(n * 20), the
    # power law unchanged below the cap
    n = 1_000_000
    w = synth.expected_degrees(n, 20.0, 2.1)
    cap = np.sqrt(n * 20.0)
    assert w.max() <= cap * (1 + 1e-12)
    assert abs(w.mean() - 20.0) < 1e-9
    free = w < cap * (1 - 1e-12)
    i = np.flatnonzero(free)[:1000]
    ratio = w[i] / (i + 1.0) ** (-1.0 / 1.1)
    assert np.allclose(ratio, ratio[0], rtol=1e-12)
    assert 200 < np.count_nonzero(~free) < 1000
