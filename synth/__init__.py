"""Seeded synthetic inputs shared by the CUDA path, the oracle, the tests and the benchmark.

This module only draws random graphs, labels, weights and query shapes.  It contains none of
the method's arithmetic (no intersections, bounds, thresholds, supports or rankings), so the
oracle and the CUDA path can both use it without sharing any of the computation they are
compared on.

Every generator takes an explicit seed and uses ``numpy.random.default_rng(seed)``.  Edge lists
are returned raw (int32 ``src``/``dst``): they may hold both directions, duplicates and
self-loops; consumers symmetrize, drop self-loops and deduplicate on their own.

The workloads stand in for the paper's datasets (Section 6.1, Table 2), which are not
available: a dense Erdos-Renyi graph with a planted clique for Email, a power-law Chung-Lu
graph with planted cliques for YouTube, and Graph500-style R-MAT graphs for the labelled
CiteSeer/MiCo/Patents workloads.
"""
from __future__ import annotations

import hashlib
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "Graph", "Query", "er_planted", "chung_lu_planted", "expected_degrees", "rmat", "labels_uniform",
    "labels_zipf", "weights_uniform", "edge_weights_uniform", "random_query", "query_batch", "er_small",
    "fixture_clique_example", "fixture_pattern_example", "path_query", "cycle_query",
    "star_query", "tree_query", "serving_requests", "workload",
]


@dataclass
class Graph:
    """A raw undirected graph: ``n`` vertices and ``m`` (possibly duplicated) edges."""
    n: int
    src: np.ndarray            # int32 [m]
    dst: np.ndarray            # int32 [m]
    labels: np.ndarray | None = None   # uint8 [n]
    weights: np.ndarray | None = None  # int32 [n]
    planted: list = field(default_factory=list)  # planted cliques (sorted int lists)
    name: str = ""
    edge_weights: np.ndarray | None = None  # int32 [m]: one weight per input pair

    @property
    def m(self) -> int:
        return int(self.src.shape[0])

    def sha256(self) -> str:
        h = hashlib.sha256()
        h.update(np.int64(self.n).tobytes())
        h.update(np.ascontiguousarray(self.src, dtype=np.int32).tobytes())
        h.update(np.ascontiguousarray(self.dst, dtype=np.int32).tobytes())
        if self.labels is not None:
            h.update(np.ascontiguousarray(self.labels, dtype=np.uint8).tobytes())
        if self.weights is not None:
            h.update(np.ascontiguousarray(self.weights, dtype=np.int32).tobytes())
        if self.edge_weights is not None:
            h.update(b"edge_weights")
            h.update(np.ascontiguousarray(self.edge_weights, dtype=np.int32).tobytes())
        return h.hexdigest()


@dataclass
class Query:
    """A connected, vertex-labelled query graph with ``nq`` <= 8 vertices."""
    nq: int
    labels: list
    edges: list      # list of (a, b) pairs, a != b
    kind: str = ""

    def as_arrays(self):
        e = np.asarray(self.edges, dtype=np.int32).reshape(-1, 2)
        return (np.asarray(self.labels, dtype=np.uint8),
                np.ascontiguousarray(e[:, 0]), np.ascontiguousarray(e[:, 1]))


def _pairs_from_upper_index(idx: np.ndarray, n: int):
    """Map linear indices of the strict upper triangle (row-major) to (i, j) pairs."""
    # row i starts at offset i*n - i*(i+1)/2 ; solve for i with a float guess then fix up.
    idx = idx.astype(np.int64)
    nn = np.float64(n)
    i = np.floor(nn - 0.5 - np.sqrt((nn - 0.5) ** 2 - 2.0 * idx)).astype(np.int64)
    i = np.clip(i, 0, n - 2)
    start = i * n - i * (i + 1) // 2
    # fix rounding in both directions
    over = idx < start
    while np.any(over):
        i[over] -= 1
        start = i * n - i * (i + 1) // 2
        over = idx < start
    nxt = (i + 1) * n - (i + 1) * (i + 2) // 2
    under = idx >= nxt
    while np.any(under):
        i[under] += 1
        start = i * n - i * (i + 1) // 2
        nxt = (i + 1) * n - (i + 1) * (i + 2) // 2
        under = idx >= nxt
    j = idx - start + i + 1
    return i, j


def er_small(n: int, p: float, seed: int) -> Graph:
    """G(n, p): every pair i<j kept independently with probability p (one uniform per pair)."""
    rng = np.random.default_rng(seed)
    total = n * (n - 1) // 2
    if total == 0:
        return Graph(n, np.zeros(0, np.int32), np.zeros(0, np.int32), name=f"er{n}")
    keep = np.flatnonzero(rng.random(total) < p)
    i, j = _pairs_from_upper_index(keep, n)
    return Graph(n, i.astype(np.int32), j.astype(np.int32), name=f"er{n}_p{p}_s{seed}")


def er_planted(n: int = 2000, p: float = 0.01, clique: int = 12, seed: int = 0) -> Graph:
    """Erdos-Renyi G(n, p) plus one planted clique on ``rng.choice(n, clique)`` vertices.

    Pairs are drawn by geometric skipping (gap ~ Geometric(p) between kept pair indices), so
    the cost is proportional to the number of kept edges.
    """
    rng = np.random.default_rng(seed)
    total = n * (n - 1) // 2
    kept = []
    pos = -1
    # draw gaps in blocks until the triangle is exhausted
    while True:
        gaps = rng.geometric(p, size=max(1024, int(total * p * 1.2) + 16))
        idx = pos + np.cumsum(gaps)
        idx = idx[idx < total]
        if idx.size:
            kept.append(idx)
            pos = int(idx[-1])
        if idx.size < gaps.size:
            break
    keep = np.concatenate(kept) if kept else np.zeros(0, np.int64)
    i, j = _pairs_from_upper_index(keep, n)
    c = np.sort(rng.choice(n, clique, replace=False))
    ci, cj = np.triu_indices(clique, 1)
    src = np.concatenate([i, c[ci]]).astype(np.int32)
    dst = np.concatenate([j, c[cj]]).astype(np.int32)
    return Graph(n, src, dst, planted=[c.tolist()], name=f"er{n}_p{p}_planted{clique}_s{seed}")


def expected_degrees(n: int, mean_deg: float, beta: float) -> np.ndarray:
    """Chung-Lu expected degrees: w_i proportional to (i+1)^(-1/(beta-1)), mean ``mean_deg``,
    every weight at most sqrt(n * mean_deg).  Weights that pass the cap are pinned to it and
    the rest are rescaled to keep the mean; this repeats until no free weight passes the cap."""
    w = (np.arange(n, dtype=np.float64) + 1.0) ** (-1.0 / (beta - 1.0))
    cap = np.sqrt(n * mean_deg)
    clipped = np.zeros(n, dtype=bool)
    for _ in range(64):
        free = ~clipped
        w[free] *= (mean_deg * n - cap * clipped.sum()) / w[free].sum()
        over = free & (w > cap)
        if not over.any():
            break
        w[over] = cap
        clipped |= over
    return w


def chung_lu_planted(n: int = 1_000_000, mean_deg: float = 20.0, beta: float = 2.1,
                     n_cliques: int = 50, size_lo: int = 15, size_hi: int = 30,
                     seed: int = 0) -> Graph:
    """Chung-Lu power-law graph with vertex-disjoint planted cliques.

    Expected-degree weights w_i = (i+1)^(-1/(beta-1)) are scaled to mean ``mean_deg`` and
    clipped at sqrt(n * mean_deg): weights above the cap are set to it and only the unclipped
    ones are rescaled, repeatedly, until the mean is ``mean_deg`` and no weight exceeds the
    cap (``expected_degrees``).  n*mean_deg/2 edges are drawn with both endpoints i.i.d.
    proportional to w (inverse-CDF sampling), then the vertex ids are randomly permuted.
    Clique sizes are ``rng.integers(size_lo, size_hi + 1)``; members are disjoint, uniform.
    """
    rng = np.random.default_rng(seed)
    w = expected_degrees(n, mean_deg, beta)
    cdf = np.cumsum(w)
    cdf /= cdf[-1]
    m = int(n * mean_deg / 2)
    src = np.searchsorted(cdf, rng.random(m), side="right").astype(np.int64)
    dst = np.searchsorted(cdf, rng.random(m), side="right").astype(np.int64)
    np.minimum(src, n - 1, out=src)
    np.minimum(dst, n - 1, out=dst)
    perm = rng.permutation(n)
    src = perm[src]
    dst = perm[dst]
    sizes = rng.integers(size_lo, size_hi + 1, size=n_cliques)
    members = rng.choice(n, int(sizes.sum()), replace=False)
    planted, ps, pd = [], [], []
    off = 0
    for s in sizes:
        c = np.sort(members[off:off + s])
        off += s
        planted.append(c.tolist())
        ci, cj = np.triu_indices(int(s), 1)
        ps.append(c[ci])
        pd.append(c[cj])
    src = np.concatenate([src] + ps).astype(np.int32)
    dst = np.concatenate([dst] + pd).astype(np.int32)
    return Graph(n, src, dst, planted=planted,
                 name=f"chunglu{n}_d{mean_deg}_b{beta}_c{n_cliques}_s{seed}")


def rmat(scale: int, edge_factor: int = 16, a: float = 0.57, b: float = 0.19, c: float = 0.19,
         seed: int = 0, relabel: bool = True) -> Graph:
    """R-MAT (Graph500 style, no noise): edge_factor * 2^scale draws, then a random relabelling."""
    rng = np.random.default_rng(seed)
    n = 1 << scale
    m = edge_factor * n
    src = np.zeros(m, dtype=np.int64)
    dst = np.zeros(m, dtype=np.int64)
    ab = a + b
    abc = a + b + c
    chunk = 1 << 22
    for lo in range(0, m, chunk):
        hi = min(m, lo + chunk)
        s = np.zeros(hi - lo, dtype=np.int64)
        d = np.zeros(hi - lo, dtype=np.int64)
        for lev in range(scale):
            r = rng.random(hi - lo)
            sbit = r >= ab
            dbit = ((r >= a) & (r < ab)) | (r >= abc)
            s |= sbit.astype(np.int64) << lev
            d |= dbit.astype(np.int64) << lev
        src[lo:hi] = s
        dst[lo:hi] = d
    if relabel:
        perm = rng.permutation(n)
        src = perm[src]
        dst = perm[dst]
    return Graph(n, src.astype(np.int32), dst.astype(np.int32),
                 name=f"rmat{scale}_ef{edge_factor}_s{seed}")


def labels_uniform(n: int, num_labels: int, seed: int) -> np.ndarray:
    return np.random.default_rng(seed).integers(0, num_labels, size=n).astype(np.uint8)


def labels_zipf(n: int, num_labels: int, s: float, seed: int) -> np.ndarray:
    """Label r-1 drawn with probability proportional to r^-s, r = 1..num_labels."""
    p = np.arange(1, num_labels + 1, dtype=np.float64) ** (-s)
    p /= p.sum()
    return np.random.default_rng(seed).choice(num_labels, size=n, p=p).astype(np.uint8)


def weights_uniform(n: int, lo: int, hi: int, seed: int) -> np.ndarray:
    """Integer weights uniform on the inclusive range [lo, hi]."""
    return np.random.default_rng(seed).integers(lo, hi + 1, size=n).astype(np.int32)


def edge_weights_uniform(m: int, lo: int, hi: int, seed: int) -> np.ndarray:
    """One int32 weight per input pair, uniform in [lo, hi]."""
    return np.random.default_rng(seed).integers(lo, hi + 1, size=m).astype(np.int32)


def path_query(labels) -> Query:
    k = len(labels)
    return Query(k, list(labels), [(i, i + 1) for i in range(k - 1)], "path")


def cycle_query(labels) -> Query:
    k = len(labels)
    return Query(k, list(labels), [(i, (i + 1) % k) for i in range(k)], "cycle")


def star_query(labels) -> Query:
    k = len(labels)
    return Query(k, list(labels), [(0, i) for i in range(1, k)], "star")


def tree_query(labels, rng) -> Query:
    """Uniform random labelled tree from a Pruefer sequence."""
    k = len(labels)
    if k <= 2:
        return path_query(labels)
    seq = list(rng.integers(0, k, size=k - 2))
    degree = [1] * k
    for x in seq:
        degree[x] += 1
    edges = []
    for x in seq:
        for leaf in range(k):
            if degree[leaf] == 1:
                edges.append((leaf, int(x)))
                degree[leaf] -= 1
                degree[x] -= 1
                break
    rest = [v for v in range(k) if degree[v] == 1]
    edges.append((rest[0], rest[1]))
    return Query(k, list(labels), edges, "tree")


def random_query(rng, kind: str, size: int, num_labels: int) -> Query:
    labels = [int(x) for x in rng.integers(0, num_labels, size=size)]
    if kind == "path":
        return path_query(labels)
    if kind == "cycle":
        return cycle_query(labels)
    if kind == "star":
        return star_query(labels)
    if kind == "tree":
        return tree_query(labels, rng)
    if kind == "triangle":
        return cycle_query(labels[:3])
    raise ValueError(kind)


QUERY_KINDS = ("path", "cycle", "star", "tree")


def query_batch(count: int = 64, seed: int = 1, size_lo: int = 4, size_hi: int = 8,
                num_labels: int = 8) -> list:
    """Query i has shape QUERY_KINDS[i % 4] and a size uniform in [size_lo, size_hi]."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        size = int(rng.integers(size_lo, size_hi + 1))
        out.append(random_query(rng, QUERY_KINDS[i % 4], size, num_labels))
    return out


def serving_requests(count: int, rate: float, seed: int, num_labels: int = 8):
    """Open-loop request stream: Poisson arrivals at ``rate`` req/s, 50/50 clique / iso mix.

    Clique requests draw k uniform in 1..100; iso requests draw 3..8 vertices of one of the
    four shapes (3-vertex requests are a path or a triangle) and k uniform in 10..1000.
    Returns a list of dicts with ``t`` (arrival time, s), ``kind``, ``k`` and ``query``.
    """
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate, size=count))
    reqs = []
    for i in range(count):
        if rng.random() < 0.5:
            reqs.append({"t": float(t[i]), "kind": "clique", "k": int(rng.integers(1, 101)),
                         "query": None})
        else:
            size = int(rng.integers(3, 9))
            if size == 3:
                kind = "path" if rng.random() < 0.5 else "triangle"
            else:
                kind = QUERY_KINDS[int(rng.integers(0, 4))]
            q = random_query(rng, kind, size, num_labels)
            reqs.append({"t": float(t[i]), "kind": "iso", "k": int(rng.integers(10, 1001)),
                         "query": q})
    return reqs


def fixture_clique_example() -> Graph:
    """The 4-vertex graph of the clique example (Section 2, Figs. 1a-3), 0-based ids.

    Vertices v1..v4 -> 0..3, edges {v1v2, v1v3, v2v3, v3v4}: 9 cliques of sizes 1-3,
    P_{s1} = {v2, v3} and P_{s2} = {v3} as Section 3.2 states.
    """
    e = np.array([(0, 1), (0, 2), (1, 2), (2, 3)], dtype=np.int32)
    return Graph(4, e[:, 0].copy(), e[:, 1].copy(), name="fig1a")


def fixture_pattern_example() -> Graph:
    """The 5-vertex labelled graph of the pattern / isomorphism examples (Fig. 1b), 0-based.

    v1..v5 -> 0..4 with labels (a, b, b, b, a) -> (0, 1, 1, 1, 0) and edges
    {v1v2, v2v3, v3v4, v2v4, v5v4}.  Edge v2v4 is inferred from the supports the paper states.
    """
    e = np.array([(0, 1), (1, 2), (2, 3), (1, 3), (4, 3)], dtype=np.int32)
    lab = np.array([0, 1, 1, 1, 0], dtype=np.uint8)
    w = np.array([1, 3, 2, 3, 1], dtype=np.int32)   # = vertex degrees of this graph
    return Graph(5, e[:, 0].copy(), e[:, 1].copy(), labels=lab, weights=w, name="fig1b")


def workload(name: str) -> Graph:
    """The five named workloads, built from their stated seeds."""
    if name == "er2000":
        return er_planted(2000, 0.01, 12, seed=0)
    if name == "chunglu1m":
        return chung_lu_planted(1_000_000, 20.0, 2.1, 50, 15, 30, seed=0)
    if name == "rmat20":
        g = rmat(20, 16, seed=0)
        g.labels = labels_uniform(g.n, 8, seed=10)
        g.weights = weights_uniform(g.n, 0, 1000, seed=11)
        g.name = "rmat20_l8_w1000"
        return g
    if name == "rmat18z":
        g = rmat(18, 16, seed=0)
        g.labels = labels_zipf(g.n, 16, 1.2, seed=10)
        g.name = "rmat18_zipf16"
        return g
    if name == "rmat22":
        g = rmat(22, 16, seed=0)
        g.labels = labels_uniform(g.n, 8, seed=10)
        g.weights = weights_uniform(g.n, 0, 1000, seed=11)
        g.name = "rmat22_l8_w1000"
        return g
    raise KeyError(name)
