"""Brute force from the definitions, for tiny graphs -- TEST INFRASTRUCTURE ONLY.

Pure Python, no pruning, no priorities: every object is enumerated and ranked afterwards.
Used to pin the Algorithm 1 / Algorithm 2 oracle (``nuri_oracle.cpp``) on small inputs.

* cliques: every non-empty pairwise-adjacent vertex set (Section 2 "Clique Discovery"),
  score = size (or the sum of vertex weights); CLIQUE_MAXIMAL keeps the ones no vertex can
  extend.
* subgraph isomorphism: every injective label-preserving map of the query whose query edges
  land on data edges (Section 2 "Subgraph Isomorphism", non-induced reading); a result is the
  image (V_s, E_s); score = sum of vertex scores, or of edge weights over E_s.
* patterns: every connected M-edge subset of E defines a pattern (its image graph); a
  pattern's domains come from every injective map of the pattern into G; f = min domain size
  (Section 2, minimum image-based support).
"""
from __future__ import annotations

import itertools


def clean_adj(g):
    adj = [set() for _ in range(g.n)]
    for a, b in zip(g.src.tolist(), g.dst.tolist()):
        if a != b:
            adj[a].add(b)
            adj[b].add(a)
    return adj


def all_cliques(g):
    adj = clean_adj(g)
    out = []

    def grow(clique, cands):
        out.append(tuple(clique))
        for v in sorted(cands):
            if v > clique[-1]:
                grow(clique + [v], {u for u in cands if u in adj[v] and u > v})

    for v in range(g.n):
        grow([v], {u for u in adj[v] if u > v})
    return out


def topk_cliques(g, k, maximal=False):
    adj = clean_adj(g)
    cl = all_cliques(g)
    if maximal:
        cl = [c for c in cl
              if not set.intersection(*[adj[v] for v in c]) - set(c)]
    cl.sort(key=lambda c: (-len(c), c))
    return [(len(c), c) for c in cl[:k]]


def topk_wcliques(g, k, maximal=False):
    """Every clique scored by the sum of its vertex weights; ties by sorted ids."""
    adj = clean_adj(g)
    w = g.weights.tolist()
    cl = all_cliques(g)
    if maximal:
        cl = [c for c in cl
              if not set.intersection(*[adj[v] for v in c]) - set(c)]
    rows = sorted(((sum(w[v] for v in c), c) for c in cl), key=lambda r: (-r[0], r[1]))
    return rows[:k]


def edge_weight_map(g):
    """Weight of each undirected edge {a, b} (a < b): the largest weight of its input pairs."""
    w = {}
    for a, b, x in zip(g.src.tolist(), g.dst.tolist(), g.edge_weights.tolist()):
        if a != b:
            e = (min(a, b), max(a, b))
            w[e] = max(w.get(e, x), x)
    return w


def iso_images(g, q, degree_rank=False, induced=False, edge_rank=False):
    """All distinct images (V_s, E_s) of matches, with their scores: non-induced (query
    edges land on data edges), or induced (also: non-adjacent query vertices land on
    non-adjacent data vertices).  Scores: sum of vertex weights or degrees over V_s, or
    (edge_rank) sum of edge weights over E_s."""
    adj = clean_adj(g)
    lab = g.labels.tolist()
    ew = edge_weight_map(g) if edge_rank else None
    if edge_rank:
        score = None
    else:
        score = [len(adj[v]) for v in range(g.n)] if degree_rank else g.weights.tolist()
    cands = [[v for v in range(g.n) if lab[v] == q.labels[i]] for i in range(q.nq)]
    images = {}
    for mp in itertools.product(*cands):
        if len(set(mp)) != q.nq:
            continue
        if all(mp[b] in adj[mp[a]] for a, b in q.edges):
            if induced:
                qe = {(min(a, b), max(a, b)) for a, b in q.edges}
                if any(mp[b] in adj[mp[a]] for a in range(q.nq) for b in range(a + 1, q.nq)
                       if (a, b) not in qe):
                    continue
            V = tuple(sorted(mp))
            E = tuple(sorted((min(mp[a], mp[b]), max(mp[a], mp[b])) for a, b in q.edges))
            images[(V, E)] = sum(ew[e] for e in E) if edge_rank else sum(score[v] for v in mp)
    return images


def topk_iso(g, q, k, degree_rank=False, induced=False, edge_rank=False):
    im = iso_images(g, q, degree_rank, induced, edge_rank)
    rows = sorted(((s, V, E) for (V, E), s in im.items()), key=lambda r: (-r[0], r[1], r[2]))
    return rows[:k]


def canon_code(nv, labels, edges):
    """min over permutations of [nv, labels in order, upper-triangle bits row-major]."""
    A = [[0] * nv for _ in range(nv)]
    for a, b in edges:
        A[a][b] = A[b][a] = 1
    best = None
    for perm in itertools.permutations(range(nv)):
        c = [nv] + [labels[perm[j]] for j in range(nv)]
        c += [A[perm[a]][perm[b]] for a in range(nv) for b in range(a + 1, nv)]
        c = tuple(c)
        if best is None or c < best:
            best = c
    return best


def pattern_mni(g, nv, labels, edges):
    """Domains from every injective, label- and edge-preserving map (non-induced)."""
    adj = clean_adj(g)
    lab = g.labels.tolist()
    cands = [[v for v in range(g.n) if lab[v] == labels[i]] for i in range(nv)]
    dom = [set() for _ in range(nv)]
    for mp in itertools.product(*cands):
        if len(set(mp)) != nv:
            continue
        if all(mp[b] in adj[mp[a]] for a, b in edges):
            for i in range(nv):
                dom[i].add(mp[i])
    return min(len(d) for d in dom), [len(d) for d in dom]


def _connected(edges):
    vs = {x for e in edges for x in e}
    if not vs:
        return False
    start = next(iter(vs))
    seen = {start}
    stack = [start]
    while stack:
        a = stack.pop()
        for x, y in edges:
            for u, v in ((x, y), (y, x)):
                if u == a and v not in seen:
                    seen.add(v)
                    stack.append(v)
    return seen == vs


def topk_patterns(g, M, k):
    """Patterns = image graphs of connected M-edge subsets of E; ranked by (f desc, code asc)."""
    adj = clean_adj(g)
    lab = g.labels.tolist()
    E = sorted({(min(a, b), max(a, b)) for a in range(g.n) for b in adj[a]})
    pats = {}
    for sub in itertools.combinations(E, M):
        if not _connected(sub):
            continue
        vs = sorted({x for e in sub for x in e})
        pos = {v: i for i, v in enumerate(vs)}
        labels = [lab[v] for v in vs]
        pe = [(pos[a], pos[b]) for a, b in sub]
        code = canon_code(len(vs), labels, pe)
        if code not in pats:
            pats[code] = (len(vs), labels, pe)
    rows = []
    for code, (nv, labels, pe) in pats.items():
        f, _ = pattern_mni(g, nv, labels, pe)
        rows.append((f, code))
    rows.sort(key=lambda r: (-r[0], r[1]))
    return rows[:k]


def code_from_row(nv, labels, edges):
    return canon_code(nv, list(labels), list(edges))
