"""The oracle -- TEST INFRASTRUCTURE ONLY.

Plain, slow CPU implementations of what the paper's method computes, used to check the CUDA
library: only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py``
may import this package.  It shares no code with the CUDA path.

* ``nuri_oracle.cpp`` (built here into ``liboracle.so`` with g++): Algorithm 1 for cliques and
  subgraph isomorphism, Algorithm 2 for patterns, Bron-Kerbosch, the hop/label index, MNI.
* ``brute.py``: brute force straight from the definitions for tiny graphs.

Python-side results are lists of rows ``(score, verts, edges, labels)``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "nuri_oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile liboracle.so next to its source (g++, -O2)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


class _Res(ctypes.Structure):
    _fields_ = [
        ("count", ctypes.c_int32),
        ("score", ctypes.POINTER(ctypes.c_int64)),
        ("vert_off", ctypes.POINTER(ctypes.c_int32)),
        ("verts", ctypes.POINTER(ctypes.c_int32)),
        ("edge_off", ctypes.POINTER(ctypes.c_int32)),
        ("edges", ctypes.POINTER(ctypes.c_int32)),
        ("labels", ctypes.POINTER(ctypes.c_int32)),
        ("expansions", ctypes.c_int64),
        ("dequeued", ctypes.c_int64),
        ("pruned", ctypes.c_int64),
        ("complete", ctypes.c_int32),
        ("seconds", ctypes.c_double),
    ]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            P = ctypes.c_void_p
            i32, i64 = ctypes.c_int32, ctypes.c_int64
            RP = ctypes.POINTER(ctypes.POINTER(_Res))
            L.orc_free.argtypes = [ctypes.POINTER(_Res)]
            L.orc_topk_cliques.argtypes = [i32, i64, P, P, i32, i32, i64, RP]
            L.orc_bk_cliques.argtypes = [i32, i64, P, P, i32, i32, RP]
            L.orc_topk_wcliques.argtypes = [i32, i64, P, P, P, i32, i32, i64, RP]
            L.orc_hop_index.argtypes = [i32, i64, P, P, P, P, i32, i32, i32, P]
            L.orc_topk_iso.argtypes = [i32, i64, P, P, P, P, P, i32, i32, P, i32, P, P, i32,
                                       i64, i32, RP]
            L.orc_mni.argtypes = [i32, i64, P, P, P, i32, P, i32, P, P, P, P]
            L.orc_topk_patterns.argtypes = [i32, i64, P, P, P, i32, i32, RP]
            L.orc_canonical_code.argtypes = [i32, P, i32, P, P, P, P]
            _lib = L
    return _lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


class Result(list):
    """Rows ``(score, verts, edges, labels)`` plus the run's counters."""
    expansions = 0
    dequeued = 0
    pruned = 0
    complete = True
    seconds = 0.0


def _unpack(rp) -> Result:
    r = rp.contents
    out = Result()
    for i in range(r.count):
        v0, v1 = r.vert_off[i], r.vert_off[i + 1]
        e0, e1 = r.edge_off[i], r.edge_off[i + 1]
        verts = tuple(r.verts[j] for j in range(v0, v1))
        labels = tuple(r.labels[j] for j in range(v0, v1))
        edges = tuple((r.edges[2 * j], r.edges[2 * j + 1]) for j in range(e0, e1))
        out.append((int(r.score[i]), verts, edges, labels))
    out.expansions, out.dequeued, out.pruned = r.expansions, r.dequeued, r.pruned
    out.complete, out.seconds = bool(r.complete), r.seconds
    lib().orc_free(rp)
    return out


def _edges(g):
    return (np.ascontiguousarray(g.src, dtype=np.int32),
            np.ascontiguousarray(g.dst, dtype=np.int32))


def topk_cliques(g, k: int, maximal: bool = False, budget: int = 0) -> Result:
    """Algorithm 1 with the clique functions of Section 3.2 (ids as canonical order)."""
    s, d = _edges(g)
    rp = ctypes.POINTER(_Res)()
    rc = lib().orc_topk_cliques(g.n, s.size, _ptr(s), _ptr(d), k, int(maximal), budget,
                                ctypes.byref(rp))
    if rc:
        raise ValueError("orc_topk_cliques rc=%d" % rc)
    return _unpack(rp)


def topk_wcliques(g, k: int, maximal: bool = False, budget: int = 0) -> Result:
    """Algorithm 1 with the clique functions, ranked by the sum of ``g.weights`` over the
    clique (Section 2's top-k semantics with a cumulative weight)."""
    s, d = _edges(g)
    w = np.ascontiguousarray(g.weights, dtype=np.int32)
    rp = ctypes.POINTER(_Res)()
    rc = lib().orc_topk_wcliques(g.n, s.size, _ptr(s), _ptr(d), _ptr(w), k, int(maximal),
                                 budget, ctypes.byref(rp))
    if rc:
        raise ValueError("orc_topk_wcliques rc=%d" % rc)
    return _unpack(rp)


def bk_cliques(g, k: int, maximal: bool) -> Result:
    """Bron-Kerbosch (pivoting, degeneracy order): top-k maximal, or all via subsets."""
    s, d = _edges(g)
    rp = ctypes.POINTER(_Res)()
    rc = lib().orc_bk_cliques(g.n, s.size, _ptr(s), _ptr(d), k, int(maximal), ctypes.byref(rp))
    if rc:
        raise ValueError("orc_bk_cliques rc=%d" % rc)
    return _unpack(rp)


def hop_index(g, num_labels: int, hops: int, method: int = 1) -> np.ndarray:
    """index[h-1, v, l] (Section 4.3 / Listing 3, cumulative hops); -1 = no such vertex."""
    s, d = _edges(g)
    lab = np.ascontiguousarray(g.labels, dtype=np.uint8)
    w = np.ascontiguousarray(g.weights, dtype=np.int32)
    out = np.empty((hops, g.n, num_labels), dtype=np.int32)
    rc = lib().orc_hop_index(g.n, s.size, _ptr(s), _ptr(d), _ptr(lab), _ptr(w), num_labels,
                             hops, method, _ptr(out))
    if rc:
        raise ValueError("orc_hop_index rc=%d" % rc)
    return out


def topk_iso(g, q, k: int, degree_rank: bool = False, budget: int = 0,
             induced: bool = False, edge_rank: bool = False) -> Result:
    """Algorithm 1 with the subgraph-isomorphism functions of Section 4.3 (induced: the
    images of non-adjacent query vertices must be non-adjacent too; edge_rank: scores are
    sums of ``g.edge_weights`` over the image's edges, Section 2's cumulative edge weight)."""
    s, d = _edges(g)
    lab = np.ascontiguousarray(g.labels, dtype=np.uint8)
    w = None if g.weights is None else np.ascontiguousarray(g.weights, dtype=np.int32)
    ew = None if g.edge_weights is None else np.ascontiguousarray(g.edge_weights, dtype=np.int32)
    rank = 2 if edge_rank else (1 if degree_rank else 0)
    ql, qs, qd = q.as_arrays()
    rp = ctypes.POINTER(_Res)()
    rc = lib().orc_topk_iso(g.n, s.size, _ptr(s), _ptr(d), _ptr(lab), _ptr(w), _ptr(ew),
                            rank, q.nq, _ptr(ql), qs.size, _ptr(qs), _ptr(qd), k,
                            budget, int(induced), ctypes.byref(rp))
    if rc:
        raise ValueError("orc_topk_iso rc=%d" % rc)
    return _unpack(rp)


def mni(g, plabels, pedges):
    """Minimum image-based support of a pattern and its per-vertex domain sizes."""
    s, d = _edges(g)
    lab = np.ascontiguousarray(g.labels, dtype=np.uint8)
    pl = np.ascontiguousarray(plabels, dtype=np.int32)
    pe = np.asarray(pedges, dtype=np.int32).reshape(-1, 2)
    ps, pd = np.ascontiguousarray(pe[:, 0]), np.ascontiguousarray(pe[:, 1])
    f = np.zeros(1, np.int64)
    dom = np.zeros(pl.size, np.int64)
    rc = lib().orc_mni(g.n, s.size, _ptr(s), _ptr(d), _ptr(lab), pl.size, _ptr(pl), ps.size,
                       _ptr(ps), _ptr(pd), _ptr(f), _ptr(dom))
    if rc:
        raise ValueError("orc_mni rc=%d" % rc)
    return int(f[0]), dom.tolist()


def topk_patterns(g, M: int, k: int) -> Result:
    """Algorithm 2 with the pattern-mining functions of Section 4.2 (MNI support)."""
    s, d = _edges(g)
    lab = np.ascontiguousarray(g.labels, dtype=np.uint8)
    rp = ctypes.POINTER(_Res)()
    rc = lib().orc_topk_patterns(g.n, s.size, _ptr(s), _ptr(d), _ptr(lab), M, k,
                                 ctypes.byref(rp))
    if rc:
        raise ValueError("orc_topk_patterns rc=%d" % rc)
    return _unpack(rp)


def canonical_code(plabels, pedges):
    """Canonical code [n, labels..., upper-triangle bits...] and the permutation reaching it."""
    pl = np.ascontiguousarray(plabels, dtype=np.int32)
    pe = np.asarray(pedges, dtype=np.int32).reshape(-1, 2)
    ps, pd = np.ascontiguousarray(pe[:, 0]), np.ascontiguousarray(pe[:, 1])
    n = pl.size
    code = np.zeros(1 + n + n * (n - 1) // 2, np.int32)
    perm = np.zeros(n, np.int32)
    rc = lib().orc_canonical_code(n, _ptr(pl), ps.size, _ptr(ps), _ptr(pd), _ptr(code),
                                  _ptr(perm))
    if rc:
        raise ValueError("orc_canonical_code rc=%d" % rc)
    return tuple(int(x) for x in code), perm.tolist()
