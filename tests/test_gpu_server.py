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
