"""Continuous-batching server: every result equals the same query run alone (and the oracle),
requests arriving together are merged into batched launches, errors stay per request."""
import numpy as np
import pytest

import oracle
import synth

nuri = pytest.importorskip("paper_1807_08888_b300")
pytestmark = pytest.mark.gpu


def _graph():
    g = synth.rmat(11, 16, seed=61)
    g.labels = synth.labels_uniform(g.n, 8, seed=62)
    g.weights = synth.weights_uniform(g.n, 0, 1000, seed=63)
    return g


def test_mix_equals_alone_and_oracle():
    g = _graph()
    G = nuri.load_graph(g.n, g.src, g.dst, labels=g.labels, weights=g.weights, index_hops=4)
    reqs = synth.serving_requests(80, rate=1e9, seed=5)  # all arrive at once
    srv = nuri.Server(G, slots=4, max_batch=16)
    tickets = []
    for r in reqs:
        if r["kind"] == "clique":
            tickets.append(srv.submit_cliques(r["k"]))
        else:
            tickets.append(srv.submit_iso(r["query"], r["k"]))
    outs = [srv.wait(t) for t in tickets]
    st = srv.stats()
    srv.close()
    n_iso = sum(r["kind"] == "iso" for r in reqs)
    assert st["iso_batched_requests"] == n_iso
    assert st["iso_batches"] < n_iso  # some requests shared a launch
    n_cl = len(reqs) - n_iso
    assert st["clique_requests"] == n_cl
    assert st["clique_searches"] < n_cl  # some clique requests shared a search
    for r, (res, times) in zip(reqs, outs):
        assert times["total_ms"] >= times["service_ms"] >= 0
        if r["kind"] == "clique":
            alone = nuri.topk_cliques(G, r["k"])
            assert [(x[0], x[1]) for x in res] == [(x[0], x[1]) for x in alone]
        else:
            alone = nuri.topk_iso(G, r["query"], r["k"])
            assert [tuple(x) for x in res] == [tuple(x) for x in alone]
    # oracle on a sample
    for r, (res, _) in list(zip(reqs, outs))[:12]:
        if r["kind"] == "iso":
            want = [(x[0], tuple(x[1]), tuple(x[2])) for x in oracle.topk_iso(g, r["query"], r["k"])]
            assert [tuple(x) for x in res] == want


def test_poll_pending_and_request_errors():
    g = _graph()
    G = nuri.load_graph(g.n, g.src, g.dst, labels=g.labels, weights=g.weights, index_hops=2)
    srv = nuri.Server(G, slots=2)
    bad = synth.Query(3, [0, 1, 2], [(0, 1)])  # disconnected: rejected at submission
    with pytest.raises(nuri.NuriError):
        srv.submit_iso(bad, 5)
    t_ok = srv.submit_cliques(3)
    t_iso = srv.submit_iso(synth.path_query([1, 2, 3]), 5)
    res, _ = srv.wait(t_ok)
    res_iso, _ = srv.wait(t_iso)
    assert [tuple(x) for x in res_iso] == [tuple(x) for x in nuri.topk_iso(G, synth.path_query([1, 2, 3]), 5)]
    assert [(x[0], x[1]) for x in res] == [(x[0], x[1]) for x in nuri.topk_cliques(G, 3)]
    # a finished ticket is reported once
    with pytest.raises(nuri.NuriError):
        srv.poll(t_ok)
    srv.close()


def test_memory_admission_serialises_clique_requests():
    """Admission by device memory: with a budget below two clique requests' footprint (the
    upper bound nuri_request_bytes gives, plus the memory held for the whole run), two clique
    requests submitted together run one after the other; with room for both they may
    overlap.  Results are the same as alone either way."""
    g = synth.chung_lu_planted(20000, 20.0, 2.1, 10, 8, 16, seed=5)
    G = nuri.load_graph(g.n, g.src, g.dst)
    foot = nuri.request_bytes(G, "clique", 50)
    assert foot > 0
    alone = [(x[0], x[1]) for x in nuri.topk_cliques(G, 50)]
    probe = nuri.Server(G, slots=2)
    _, fixed = probe.budget()
    probe.close()
    # max_batch=1: the two requests may not share one search
    srv = nuri.Server(G, slots=2, max_batch=1, mem_budget_bytes=fixed + int(1.5 * foot))
    assert srv.budget() == (fixed + int(1.5 * foot), fixed)
    t1 = srv.submit_cliques(50)
    t2 = srv.submit_cliques(50)
    (r1, m1), (r2, m2) = srv.wait(t1), srv.wait(t2)
    srv.close()
    assert [(x[0], x[1]) for x in r1] == alone and [(x[0], x[1]) for x in r2] == alone
    assert m1["mem_bytes"] == foot and m2["mem_bytes"] == foot
    first, second = sorted([m1, m2], key=lambda m: m["start_ms"])
    assert second["start_ms"] >= first["done_ms"]  # no overlap: admitted one at a time
    assert second["queue_ms"] > 0


def test_topk_batch_mixed_kinds_equal_alone_and_oracle():
    """nuri_topk_batch over cliques (all and maximal, with and without kept ties), isomorphism
    queries and patterns: every request's rows equal the request run alone and the oracle."""
    g = _graph()
    G = nuri.load_graph(g.n, g.src, g.dst, labels=g.labels, weights=g.weights, index_hops=4)
    qs = synth.query_batch(6, seed=8, size_lo=3, size_hi=6, num_labels=8)
    reqs = [("clique", 1), ("clique", 37), ("iso", qs[0], 10), ("clique", 5),
            ("clique", 10, True), ("clique", 3, False, True), ("patterns", 2, 5),
            ("iso", qs[1], 100), ("clique", 100), ("patterns", 3, 10), ("patterns", 2, 1),
            ("iso", qs[2], 7, True)] + [("iso", q, 50) for q in qs[3:]]
    out = nuri.topk_batch(G, reqs)
    assert len(out) == len(reqs)
    for r, got in zip(reqs, out):
        rows = [tuple(x) for x in got]
        if r[0] == "clique":
            maximal = len(r) > 2 and r[2]
            ties = len(r) > 3 and r[3]
            alone = nuri.topk_cliques(G, r[1], maximal=maximal, keep_ties=ties)
            assert rows == [tuple(x) for x in alone], r
            if not ties:
                want = [(x[0], tuple(x[1])) for x in oracle.topk_cliques(g, r[1], maximal)]
                assert rows == want, r
        elif r[0] == "iso":
            deg = len(r) > 3 and r[3]
            alone = nuri.topk_iso(G, r[1], r[2], degree_rank=deg)
            assert rows == [tuple(x) for x in alone]
            want = [(x[0], tuple(x[1]), tuple(x[2])) for x in oracle.topk_iso(g, r[1], r[2], deg)]
            assert rows == want
        else:
            alone = nuri.topk_patterns(G, r[1], r[2])
            assert rows == [tuple(x) for x in alone]
            want = [(x[0], tuple(x[3]), tuple(x[2])) for x in oracle.topk_patterns(g, r[1], r[2])]
            assert rows == want
    # a bad request fails the call and returns nothing
    with pytest.raises(nuri.NuriError):
        nuri.topk_batch(G, [("clique", 3), ("patterns", 6, 1)])
