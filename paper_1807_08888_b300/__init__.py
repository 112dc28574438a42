"""Python binding of libnuri (C ABI in include/nuri.h): argument marshalling only.

Every step of a query runs inside libnuri's CUDA kernels; this module converts arrays to
pointers, calls the C entry points and turns the library-owned result into Python rows.
There is no CPU fallback: if ``libnuri.so`` is missing or fails to load, every call raises.

    import paper_1807_08888_b300 as nuri
    g = nuri.load_graph(n, src, dst, labels=None, weights=None, index_hops=0)
    rows = nuri.topk_cliques(g, k=10)             # [(size, (ids...)), ...]
    rows = nuri.topk_iso(g, query, k=1000)        # [(score, (ids...), ((a,b),...)), ...]
    rows = nuri.topk_patterns(g, M=3, k=10)       # [(support, (labels...), ((i,j),...)), ...]
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

__all__ = [
    "NuriError", "lib", "load_graph", "Graph", "topk_cliques", "topk_iso", "topk_iso_batch",
    "topk_patterns", "hop_index", "hop_index_noalloc", "set_time_budget", "tune_cliques", "Server",
    "request_bytes", "topk_batch", "Result", "LIB_PATH", "EXPORTS",
    "RANK_SIZE", "RANK_WEIGHT_SUM", "RANK_DEGREE_SUM", "RANK_MNI", "RANK_EDGE_WEIGHT_SUM",
]

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libnuri.so")

OK, ERR_INVALID, ERR_OOM, ERR_LIMIT, ERR_TIMEOUT, ERR_CANCELLED, ERR_CUDA, PENDING = range(8)
REQ_CLIQUES, REQ_ISO, REQ_PATTERNS = 0, 1, 2
RANK_SIZE, RANK_WEIGHT_SUM, RANK_DEGREE_SUM, RANK_MNI, RANK_EDGE_WEIGHT_SUM = range(5)
LOAD_DEVICE_INPUT, LOAD_NO_ISO = 0x1, 0x2
CLIQUE_ALL, CLIQUE_MAXIMAL = 0x0, 0x1
KEEP_TIES, NO_PRUNE, ISO_INDUCED, PATTERNS_EDGE_ORIENTED = 0x100, 0x200, 0x400, 0x800

# every function include/nuri.h declares
EXPORTS = (
    "nuri_load_graph", "nuri_free_graph", "nuri_graph_get_info", "nuri_topk_cliques",
    "nuri_topk_iso", "nuri_topk_iso_batch", "nuri_topk_patterns", "nuri_hop_index",
    "nuri_hop_index_noalloc",
    "nuri_free_result", "nuri_last_error", "nuri_version", "nuri_set_time_budget",
    "nuri_tune_cliques",
    "nuri_server_create", "nuri_server_submit", "nuri_server_poll", "nuri_server_wait",
    "nuri_server_stats", "nuri_server_budget", "nuri_server_destroy", "nuri_request_bytes",
    "nuri_topk_batch", "nuri_server_clique_stats", "nuri_set_partition", "nuri_seed_part",
    "nuri_set_edge_weights",
)


class NuriError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"nuri error {code}: {msg}")
        self.code = code


class _Stats(ctypes.Structure):
    _fields_ = [
        ("expansions", ctypes.c_int64), ("pruned", ctypes.c_int64),
        ("dequeued", ctypes.c_int64), ("spilled", ctypes.c_int64),
        ("reloaded", ctypes.c_int64), ("results_stored", ctypes.c_int64),
        ("rounds", ctypes.c_int64), ("adj_bytes", ctypes.c_int64),
        ("threshold", ctypes.c_int64), ("restarts", ctypes.c_int32), ("pad", ctypes.c_int32),
        ("device_ms", ctypes.c_double), ("launches", ctypes.c_int64),
        ("expand_launches", ctypes.c_int64), ("expand_ms", ctypes.c_double),
        ("tail_launches", ctypes.c_int64), ("tail_ms", ctypes.c_double),
        ("tail_words", ctypes.c_int64), ("dense_records", ctypes.c_int64 * 3),
        ("lex_pruned", ctypes.c_int64),
    ]


class _Result(ctypes.Structure):
    _fields_ = [
        ("count", ctypes.c_int32), ("kind", ctypes.c_int32),
        ("score", ctypes.POINTER(ctypes.c_int64)),
        ("vert_off", ctypes.POINTER(ctypes.c_int32)), ("verts", ctypes.POINTER(ctypes.c_int32)),
        ("edge_off", ctypes.POINTER(ctypes.c_int32)), ("edges", ctypes.POINTER(ctypes.c_int32)),
        ("labels", ctypes.POINTER(ctypes.c_int32)),
        ("stats", _Stats),
    ]


class _Query(ctypes.Structure):
    _fields_ = [
        ("nq", ctypes.c_int32), ("ne", ctypes.c_int32),
        ("labels", ctypes.c_void_p), ("src", ctypes.c_void_p), ("dst", ctypes.c_void_p),
    ]


class _Request(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("k", ctypes.c_int32), ("rank", ctypes.c_int32),
                ("flags", ctypes.c_uint32), ("query", _Query),
                ("pattern_edges", ctypes.c_int32), ("pad", ctypes.c_int32)]


class _ServerCfg(ctypes.Structure):
    _fields_ = [("slots", ctypes.c_int32), ("max_batch", ctypes.c_int32),
                ("mem_budget_bytes", ctypes.c_int64)]


class _Times(ctypes.Structure):
    _fields_ = [("queue_ms", ctypes.c_double), ("service_ms", ctypes.c_double),
                ("total_ms", ctypes.c_double), ("start_ms", ctypes.c_double),
                ("done_ms", ctypes.c_double), ("mem_bytes", ctypes.c_int64)]


class _Info(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int32), ("num_labels", ctypes.c_int32), ("num_edges", ctypes.c_int64),
        ("dropped", ctypes.c_int64), ("max_degree", ctypes.c_int32),
        ("max_out_degree", ctypes.c_int32), ("index_hops", ctypes.c_int32),
        ("pad", ctypes.c_int32), ("device_bytes", ctypes.c_int64),
    ]


_lock = threading.Lock()
_lib = None


def lib():
    """Load libnuri.so (raises if it is missing: there is no fallback)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise NuriError(ERR_CUDA, f"{LIB_PATH} is not built "
                                          "(python -m paper_1807_08888_b300.build)")
            L = ctypes.CDLL(LIB_PATH)
            P, i32, i64, u32 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32
            RPP = ctypes.POINTER(ctypes.POINTER(_Result))
            L.nuri_load_graph.argtypes = [i32, i64, P, P, P, P, i32, u32, P,
                                          ctypes.POINTER(ctypes.c_void_p)]
            L.nuri_load_graph.restype = i32
            L.nuri_free_graph.argtypes = [P]
            L.nuri_free_graph.restype = None
            L.nuri_graph_get_info.argtypes = [P, ctypes.POINTER(_Info)]
            L.nuri_graph_get_info.restype = i32
            L.nuri_set_edge_weights.argtypes = [P, i64, P, P, P, u32, P]
            L.nuri_set_edge_weights.restype = i32
            L.nuri_topk_cliques.argtypes = [P, i32, i32, u32, i64, P, RPP]
            L.nuri_topk_cliques.restype = i32
            L.nuri_topk_iso.argtypes = [P, ctypes.POINTER(_Query), i32, i32, u32, P, RPP]
            L.nuri_topk_iso.restype = i32
            L.nuri_topk_iso_batch.argtypes = [P, i32, ctypes.POINTER(_Query), P, i32, u32, P,
                                              ctypes.POINTER(ctypes.POINTER(_Result))]
            L.nuri_topk_iso_batch.restype = i32
            L.nuri_topk_patterns.argtypes = [P, i32, i32, i32, u32, P, RPP]
            L.nuri_topk_patterns.restype = i32
            L.nuri_hop_index.argtypes = [P, i32, i32, P, i32, P]
            L.nuri_hop_index.restype = i32
            L.nuri_hop_index_noalloc.argtypes = [i32, P, P, i64, P, i32, P, i32, P, P]
            L.nuri_hop_index_noalloc.restype = i32
            L.nuri_tune_cliques.argtypes = [P, i32, u32, P, ctypes.POINTER(i32),
                                            ctypes.POINTER(ctypes.c_double)]
            L.nuri_tune_cliques.restype = i32
            L.nuri_set_time_budget.argtypes = [ctypes.c_double]
            L.nuri_set_time_budget.restype = i32
            L.nuri_server_create.argtypes = [P, ctypes.POINTER(_ServerCfg),
                                             ctypes.POINTER(ctypes.c_void_p)]
            L.nuri_server_create.restype = i32
            L.nuri_server_submit.argtypes = [P, ctypes.POINTER(_Request),
                                             ctypes.POINTER(ctypes.c_uint64)]
            L.nuri_server_submit.restype = i32
            for nm in ("nuri_server_poll", "nuri_server_wait"):
                f = getattr(L, nm)
                f.argtypes = [P, ctypes.c_uint64, RPP, ctypes.POINTER(_Times)]
                f.restype = i32
            L.nuri_server_stats.argtypes = [P, ctypes.POINTER(ctypes.c_int64),
                                            ctypes.POINTER(ctypes.c_int64)]
            L.nuri_server_stats.restype = i32
            L.nuri_set_partition.argtypes = [P, P]
            L.nuri_set_partition.restype = i32
            L.nuri_seed_part.argtypes = [i32, i32]
            L.nuri_seed_part.restype = i32
            L.nuri_topk_batch.argtypes = [P, i32, ctypes.POINTER(_Request), P,
                                          ctypes.POINTER(ctypes.POINTER(_Result))]
            L.nuri_topk_batch.restype = i32
            L.nuri_server_clique_stats.argtypes = [P, ctypes.POINTER(ctypes.c_int64),
                                                   ctypes.POINTER(ctypes.c_int64)]
            L.nuri_server_clique_stats.restype = i32
            L.nuri_server_budget.argtypes = [P, ctypes.POINTER(ctypes.c_int64),
                                             ctypes.POINTER(ctypes.c_int64)]
            L.nuri_server_budget.restype = i32
            L.nuri_request_bytes.argtypes = [P, ctypes.POINTER(_Request),
                                             ctypes.POINTER(ctypes.c_int64)]
            L.nuri_request_bytes.restype = i32
            L.nuri_server_destroy.argtypes = [P]
            L.nuri_server_destroy.restype = None
            L.nuri_free_result.argtypes = [ctypes.POINTER(_Result)]
            L.nuri_free_result.restype = None
            L.nuri_last_error.restype = ctypes.c_char_p
            L.nuri_version.restype = ctypes.c_char_p
            _lib = L
    return _lib


def _check(rc):
    if rc != OK:
        raise NuriError(rc, lib().nuri_last_error().decode(errors="replace"))


def _stream(stream):
    if stream is not None:
        return ctypes.c_void_p(int(stream))
    try:
        import torch
        if torch.cuda.is_available() and torch.cuda.is_initialized():
            return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    except Exception:
        pass
    return ctypes.c_void_p(0)


def _host_ptr(a, dtype):
    if a is None:
        return None, None
    arr = np.ascontiguousarray(np.asarray(a), dtype=dtype)
    return arr, arr.ctypes.data_as(ctypes.c_void_p)


class Result(list):
    """Rows in rank order plus the query's device counters (``stats``, a dict)."""
    stats: dict = {}


def _unpack(rp) -> Result:
    r = rp.contents
    out = Result()
    n = r.count
    score = np.ctypeslib.as_array(r.score, shape=(max(n, 1),))[:n].copy() if n else np.zeros(0)
    voff = np.ctypeslib.as_array(r.vert_off, shape=(n + 1,)).copy()
    eoff = np.ctypeslib.as_array(r.edge_off, shape=(n + 1,)).copy()
    nvt, net = int(voff[-1]), int(eoff[-1])
    verts = np.ctypeslib.as_array(r.verts, shape=(max(nvt, 1),))[:nvt].copy()
    edges = np.ctypeslib.as_array(r.edges, shape=(max(2 * net, 2),))[:2 * net].copy()
    labels = (np.ctypeslib.as_array(r.labels, shape=(max(nvt, 1),))[:nvt].copy()
              if r.labels else None)
    for i in range(n):
        v = tuple(int(x) for x in verts[voff[i]:voff[i + 1]])
        e = tuple((int(edges[2 * j]), int(edges[2 * j + 1])) for j in range(eoff[i], eoff[i + 1]))
        if r.kind == 0:
            out.append((int(score[i]), v))
        elif r.kind == 1:
            out.append((int(score[i]), v, e))
        else:
            lab = tuple(int(x) for x in labels[voff[i]:voff[i + 1]])
            out.append((int(score[i]), lab, e))
    s = r.stats
    out.stats = {f: getattr(s, f) for f, _ in _Stats._fields_ if f != "pad"}
    out.stats["dense_records"] = list(out.stats["dense_records"])
    lib().nuri_free_result(rp)
    return out


class Graph:
    """A device-resident graph (owns a nuri_graph*)."""

    def __init__(self, handle):
        self._h = handle

    @property
    def handle(self):
        if not self._h:
            raise NuriError(ERR_INVALID, "graph already freed")
        return self._h

    def info(self) -> dict:
        inf = _Info()
        _check(lib().nuri_graph_get_info(self.handle, ctypes.byref(inf)))
        return {f: getattr(inf, f) for f, _ in _Info._fields_ if f != "pad"}

    def set_edge_weights(self, src, dst, w, stream=None):
        """One weight (>= 0) per pair (src[e], dst[e]); an edge weighs the largest weight of
        its pairs, 0 without any (host arrays or CUDA tensors)."""
        keep = []
        flags = 0
        if hasattr(src, "is_cuda") and src.is_cuda:
            flags |= LOAD_DEVICE_INPUT
            ts = [t.contiguous() for t in (src, dst, w)]
            keep += ts
            ps, pd, pw = (ctypes.c_void_p(t.data_ptr()) for t in ts)
            m = int(src.numel())
        else:
            s, ps = _host_ptr(src, np.int32)
            d, pd = _host_ptr(dst, np.int32)
            x, pw = _host_ptr(w, np.int32)
            keep += [s, d, x]
            m = int(s.size)
        _check(lib().nuri_set_edge_weights(self.handle, m, ps, pd, pw, flags, _stream(stream)))

    def free(self):
        if self._h:
            lib().nuri_free_graph(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def load_graph(n, src, dst, labels=None, weights=None, index_hops=0, flags=0,
               stream=None) -> Graph:
    """Build the device graph from an undirected edge list (host arrays or CUDA tensors)."""
    keep = []
    if hasattr(src, "is_cuda") and src.is_cuda:
        flags |= LOAD_DEVICE_INPUT
        ptrs = []
        for t in (src, dst, labels, weights):
            if t is None:
                ptrs.append(None)
            else:
                t = t.contiguous()
                keep.append(t)
                ptrs.append(ctypes.c_void_p(t.data_ptr()))
        ps, pd, pl, pw = ptrs
        m = int(src.numel())
    else:
        s, ps = _host_ptr(src, np.int32)
        d, pd = _host_ptr(dst, np.int32)
        lab, pl = _host_ptr(labels, np.uint8)
        w, pw = _host_ptr(weights, np.int32)
        keep += [s, d, lab, w]
        m = int(s.size)
    h = ctypes.c_void_p()
    _check(lib().nuri_load_graph(int(n), m, ps, pd, pl, pw, int(index_hops), int(flags),
                                 _stream(stream), ctypes.byref(h)))
    return Graph(h)


def topk_cliques(g: Graph, k: int, maximal=False, keep_ties=False, no_prune=False,
                 frontier_cap=0, stream=None, weighted=False) -> Result:
    """weighted: rank by the sum of the vertex weights (graph loaded with weights)."""
    flags = (CLIQUE_MAXIMAL if maximal else CLIQUE_ALL) | (KEEP_TIES if keep_ties else 0) | \
        (NO_PRUNE if no_prune else 0)
    rp = ctypes.POINTER(_Result)()
    rank = RANK_WEIGHT_SUM if weighted else RANK_SIZE
    _check(lib().nuri_topk_cliques(g.handle, int(k), rank, flags, int(frontier_cap),
                                   _stream(stream), ctypes.byref(rp)))
    return _unpack(rp)


def _query_struct(q, keep):
    lab = np.ascontiguousarray(q.labels, dtype=np.uint8)
    e = np.asarray(q.edges, dtype=np.int32).reshape(-1, 2)
    s, d = np.ascontiguousarray(e[:, 0]), np.ascontiguousarray(e[:, 1])
    keep += [lab, s, d]
    return _Query(int(q.nq), int(s.size), lab.ctypes.data, s.ctypes.data, d.ctypes.data)


def _iso_rank(degree_rank, edge_rank):
    if edge_rank:
        return RANK_EDGE_WEIGHT_SUM
    return RANK_DEGREE_SUM if degree_rank else RANK_WEIGHT_SUM


def topk_iso(g: Graph, q, k: int, degree_rank=False, keep_ties=False, stream=None,
             induced=False, edge_rank=False) -> Result:
    """edge_rank: rank by the sum of the image's edge weights (Graph.set_edge_weights)."""
    return topk_iso_batch(g, [q], [k], degree_rank, keep_ties, stream, induced, edge_rank)[0]


def topk_iso_batch(g: Graph, queries, ks, degree_rank=False, keep_ties=False,
                   stream=None, induced=False, edge_rank=False) -> list:
    keep = []
    nq = len(queries)
    arr = (_Query * nq)(*[_query_struct(q, keep) for q in queries])
    kk = np.ascontiguousarray(ks, dtype=np.int32)
    outs = (ctypes.POINTER(_Result) * nq)()
    rank = _iso_rank(degree_rank, edge_rank)
    flags = (KEEP_TIES if keep_ties else 0) | (ISO_INDUCED if induced else 0)
    _check(lib().nuri_topk_iso_batch(g.handle, nq, arr, kk.ctypes.data_as(ctypes.c_void_p),
                                     rank, flags, _stream(stream), outs))
    return [_unpack(outs[i]) for i in range(nq)]


def _request(req, keep):
    """A request tuple as the C struct: ("clique", k[, maximal[, keep_ties[, weighted]]]),
    ("iso", query, k[, rank[, keep_ties]]) or ("patterns", M, k[, keep_ties]); an iso rank is
    False (vertex weights), True (degrees) or "edge" (edge weights)."""
    kind = req[0]
    if kind == "clique":
        k = req[1]
        flags = (CLIQUE_MAXIMAL if len(req) > 2 and req[2] else 0) | \
            (KEEP_TIES if len(req) > 3 and req[3] else 0)
        rank = RANK_WEIGHT_SUM if len(req) > 4 and req[4] else RANK_SIZE
        return _Request(REQ_CLIQUES, int(k), rank, flags, _Query(0, 0, None, None, None),
                        0, 0)
    if kind == "iso":
        q, k = req[1], req[2]
        r = req[3] if len(req) > 3 else False
        edge = isinstance(r, str) and r == "edge"
        rank = _iso_rank(bool(r) and not edge, edge)
        flags = KEEP_TIES if len(req) > 4 and req[4] else 0
        return _Request(REQ_ISO, int(k), rank, flags, _query_struct(q, keep), 0, 0)
    if kind == "patterns":
        M, k = req[1], req[2]
        flags = KEEP_TIES if len(req) > 3 and req[3] else 0
        return _Request(REQ_PATTERNS, int(k), RANK_MNI, flags, _Query(0, 0, None, None, None),
                        int(M), 0)
    raise ValueError(kind)


def topk_batch(g: Graph, requests, stream=None) -> list:
    """Requests of any kind in one nuri_topk_batch call (see _request for the tuples)."""
    keep = []
    n = len(requests)
    arr = (_Request * max(n, 1))(*[_request(r, keep) for r in requests])
    outs = (ctypes.POINTER(_Result) * max(n, 1))()
    _check(lib().nuri_topk_batch(g.handle, n, arr, _stream(stream), outs))
    return [_unpack(outs[i]) for i in range(n)]


def topk_patterns(g: Graph, M: int, k: int, stream=None, keep_ties=False,
                  edge_oriented=False) -> Result:
    """edge_oriented: exhaustive edge-oriented expansion (the ablation beside Algorithm 2)."""
    flags = (KEEP_TIES if keep_ties else 0) | (PATTERNS_EDGE_ORIENTED if edge_oriented else 0)
    rp = ctypes.POINTER(_Result)()
    _check(lib().nuri_topk_patterns(g.handle, int(M), int(k), RANK_MNI, flags, _stream(stream),
                                    ctypes.byref(rp)))
    return _unpack(rp)


def hop_index(g: Graph, hops: int, degree_rank=False, stream=None) -> np.ndarray:
    inf = g.info()
    out = np.empty((hops, inf["n"], max(inf["num_labels"], 1)), dtype=np.int32)
    _check(lib().nuri_hop_index(g.handle, int(hops), int(bool(degree_rank)),
                                out.ctypes.data_as(ctypes.c_void_p), 0, _stream(stream)))
    return out


def hop_index_noalloc(n, off, adj, nnz, labels, L, score, hops, out, stream=None):
    """nuri_hop_index_noalloc on caller-held device arrays (raw device pointers as ints): the
    hop/label index of a CSR graph written into `out` (int32[hops * n * L]) with no device
    memory allocated by the call, for callers that cannot allocate at that point.  The library
    keeps one fixed 4 MiB scratch array per GPU for it; overlapping calls race."""
    _check(lib().nuri_hop_index_noalloc(int(n), off, adj, int(nnz), labels, int(L), score,
                                        int(hops), out, _stream(stream)))


def _times(tm):
    return {f: getattr(tm, f) for f, _ in _Times._fields_}


def request_bytes(g: Graph, kind, k, query=None, maximal=False) -> int:
    """Device bytes the server admits a request with (nuri_request_bytes); kind is
    "clique" or "iso"."""
    keep = []
    r = _request(("clique", k, maximal) if kind == "clique" else ("iso", query, k), keep)
    b = ctypes.c_int64()
    _check(lib().nuri_request_bytes(g.handle, ctypes.byref(r), ctypes.byref(b)))
    return b.value


class Server:
    """Continuous-batching request server over a resident graph (nuri_server_*)."""

    def __init__(self, g: Graph, slots=4, max_batch=64, mem_budget_bytes=0):
        """mem_budget_bytes: device memory the server admits requests into (0: the library's
        default, 80 % of the free device memory at creation)."""
        self._g = g  # keep the graph alive
        cfg = _ServerCfg(int(slots), int(max_batch), int(mem_budget_bytes))
        h = ctypes.c_void_p()
        _check(lib().nuri_server_create(g.handle, ctypes.byref(cfg), ctypes.byref(h)))
        self._h = h

    def submit_cliques(self, k, maximal=False) -> int:
        r = _request(("clique", k, maximal), [])
        t = ctypes.c_uint64()
        _check(lib().nuri_server_submit(self._h, ctypes.byref(r), ctypes.byref(t)))
        return t.value

    def submit_iso(self, q, k, degree_rank=False) -> int:
        keep = []
        r = _request(("iso", q, k, degree_rank), keep)
        t = ctypes.c_uint64()
        _check(lib().nuri_server_submit(self._h, ctypes.byref(r), ctypes.byref(t)))
        return t.value

    def budget(self):
        """(budget bytes, bytes held for the whole run)."""
        a, b = ctypes.c_int64(), ctypes.c_int64()
        _check(lib().nuri_server_budget(self._h, ctypes.byref(a), ctypes.byref(b)))
        return a.value, b.value

    def poll(self, ticket):
        """(result, times) when finished, None while pending; raises on a failed request."""
        rp = ctypes.POINTER(_Result)()
        tm = _Times()
        rc = lib().nuri_server_poll(self._h, ctypes.c_uint64(ticket), ctypes.byref(rp),
                                    ctypes.byref(tm))
        if rc == PENDING:
            return None
        _check(rc)
        return _unpack(rp), _times(tm)

    def wait(self, ticket):
        rp = ctypes.POINTER(_Result)()
        tm = _Times()
        _check(lib().nuri_server_wait(self._h, ctypes.c_uint64(ticket), ctypes.byref(rp),
                                      ctypes.byref(tm)))
        return _unpack(rp), _times(tm)

    def stats(self):
        a, b = ctypes.c_int64(), ctypes.c_int64()
        _check(lib().nuri_server_stats(self._h, ctypes.byref(a), ctypes.byref(b)))
        c, d = ctypes.c_int64(), ctypes.c_int64()
        _check(lib().nuri_server_clique_stats(self._h, ctypes.byref(c), ctypes.byref(d)))
        return {"iso_batches": a.value, "iso_batched_requests": b.value,
                "clique_searches": c.value, "clique_requests": d.value}

    def close(self):
        if self._h:
            lib().nuri_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def tune_cliques(g: Graph, k: int, maximal=False, stream=None):
    """Autotune the dense clique search on g (nuri_tune_cliques): times one top-k query per
    candidate task granularity and keeps the fastest for later queries on g.  Returns
    (chosen granularity, its device ms)."""
    c = ctypes.c_int32()
    t = ctypes.c_double()
    _check(lib().nuri_tune_cliques(g.handle, int(k), CLIQUE_MAXIMAL if maximal else 0,
                                   _stream(stream), ctypes.byref(c), ctypes.byref(t)))
    return int(c.value), float(t.value)


def set_time_budget(ms: float) -> None:
    """Limit the device time of every later query (0 = no limit); overruns raise NuriError
    with code ERR_TIMEOUT."""
    _check(lib().nuri_set_time_budget(float(ms)))


def version() -> str:
    return lib().nuri_version().decode()
