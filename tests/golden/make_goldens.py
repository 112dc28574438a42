"""Write the oracle-computed expected results the GPU parity tests compare against.

    python tests/golden/make_goldens.py [case ...]      # default: every case

Every expected value here comes from ``oracle/`` (Bron-Kerbosch, Algorithm 1 and
Algorithm 2 as the oracle restates them) run on the seeded inputs of ``synth``; nothing is
read from the CUDA library.  Each file records the recipe of its input and the SHA-256 of the
generated edge list, so a change of a generator is detected instead of silently compared.

Large row lists are stored as a digest: the SHA-256 of the rows serialised by ``row_digest``
(the tests serialise the GPU rows the same way), with the row count, the k-th score and the
first rows kept in the clear for diagnosis.
"""
from __future__ import annotations

import hashlib
import json
import multiprocessing as mp
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def row_digest(rows) -> str:
    """SHA-256 of rows given as (score, vertex tuple[, edge tuple]) in rank order."""
    canon = []
    for r in rows:
        item = [int(r[0]), [int(x) for x in r[1]]]
        if len(r) > 2:
            item.append([[int(a), int(b)] for a, b in r[2]])
        canon.append(item)
    return hashlib.sha256(json.dumps(canon, separators=(",", ":")).encode()).hexdigest()


# ---- clique graphs whose degeneracy-ordered candidate sets pass 256 (8-word tier) ----------
CLIQUE_CASES = {
    # G(1200, 0.25): degeneracy about 264, ~100 vertices with more than 256 later neighbours
    "er1200_p025_s91": ("er_small", (1200, 0.25, 91)),
    # G(1000, 0.33): degeneracy about 294, ~200 such vertices
    "er1000_p033_s5": ("er_small", (1000, 0.33, 5)),
}

# the headline recipe (Chung-Lu, mean degree 20, exponent 2.1, 50 planted cliques of 15..30)
# at sizes the Bron-Kerbosch oracle finishes (n = 1M does not: Algorithm 1 stops incomplete
# after 10^9 expansions, Bron-Kerbosch runs past half an hour on the hub block)
CHUNGLU_CASES = {
    "chunglu100k": (100_000, 20.0, 2.1, 50, 15, 30, 0),
}


def chunglu_graph(name):
    import synth
    return synth.chung_lu_planted(*CHUNGLU_CASES[name])


def make_chunglu(name, k=100):
    import oracle
    g = chunglu_graph(name)
    t = time.time()
    allr = oracle.bk_cliques(g, k, False)
    out = {"case": name, "recipe": list(CHUNGLU_CASES[name]), "sha256_graph": g.sha256(),
           "source": "oracle.bk_cliques (Bron-Kerbosch, pivoting, degeneracy order), "
                     "all-cliques ranking",
           "oracle_seconds": time.time() - t,
           "all": [[r[0], list(r[1])] for r in allr]}
    with open(os.path.join(HERE, f"cliques_{name}.json"), "w") as f:
        json.dump(out, f, separators=(",", ":"))
    print(name, out["oracle_seconds"], flush=True)


def clique_graph(name):
    import synth
    fn, args = CLIQUE_CASES[name]
    return getattr(synth, fn)(*args)


def make_cliques(name, k_all=1000, k_max=100):
    import oracle
    g = clique_graph(name)
    t = time.time()
    allr = oracle.bk_cliques(g, k_all, False)
    t_all = time.time() - t
    t = time.time()
    maxr = oracle.bk_cliques(g, k_max, True)
    t_max = time.time() - t
    # Algorithm 1 (the paper's order and bound) agrees on the top 10
    a1 = oracle.topk_cliques(g, 10)
    assert [(r[0], r[1]) for r in a1] == [(r[0], r[1]) for r in allr[:10]], name
    out = {"case": name, "recipe": list(CLIQUE_CASES[name]), "sha256_graph": g.sha256(),
           "source": "oracle.bk_cliques (Bron-Kerbosch, pivoting, degeneracy order); "
                     "top 10 also equal to oracle.topk_cliques (Algorithm 1)",
           "oracle_seconds": {"all": t_all, "maximal": t_max},
           "all": [[r[0], list(r[1])] for r in allr],
           "maximal": [[r[0], list(r[1])] for r in maxr]}
    with open(os.path.join(HERE, f"cliques_{name}.json"), "w") as f:
        json.dump(out, f, separators=(",", ":"))
    print(name, "all", t_all, "maximal", t_max, flush=True)


# ---- isomorphism: the 64 seeded queries on R-MAT 20, top-1000 each -----------------------
def _iso_one(i):
    import oracle
    import synth
    g = synth.workload("rmat20")
    q = synth.query_batch(64, seed=1)[i]
    t = time.time()
    r = oracle.topk_iso(g, q, 1000)
    rows = [(x[0], tuple(x[1]), tuple(x[2])) for x in r]
    return i, time.time() - t, rows


def make_iso_rmat20(workers=6):
    import synth
    g = synth.workload("rmat20")
    qs = synth.query_batch(64, seed=1)
    ctx = mp.get_context("spawn")
    res = {}
    with ctx.Pool(workers) as p:
        for i, sec, rows in p.imap_unordered(_iso_one, range(64)):
            res[i] = {"query": {"nq": qs[i].nq, "labels": list(qs[i].labels),
                                "edges": [list(e) for e in qs[i].edges], "kind": qs[i].kind},
                      "count": len(rows), "digest": row_digest(rows),
                      "kth_score": rows[-1][0] if rows else None,
                      "head": [[r[0], list(r[1]), [list(e) for e in r[2]]] for r in rows[:3]],
                      "oracle_seconds": sec}
            print("iso", i, sec, flush=True)
    out = {"case": "rmat20_iso64_top1000", "workload": "rmat20", "k": 1000,
           "sha256_graph": g.sha256(),
           "source": "oracle.topk_iso (Algorithm 1 with the isomorphism functions of "
                     "Section 4.3), one query at a time, weight-sum ranking",
           "queries": [res[i] for i in range(64)]}
    with open(os.path.join(HERE, "iso_rmat20_top1000.json"), "w") as f:
        json.dump(out, f, separators=(",", ":"))


# ---- patterns: R-MAT 18 with Zipf labels, M = 1..5, top-10 --------------------------------
def make_patterns_rmat18z(Ms=(1, 2, 3, 4, 5)):
    import oracle
    import synth
    g = synth.workload("rmat18z")
    out = {"case": "rmat18z_top10", "workload": "rmat18z", "k": 10,
           "sha256_graph": g.sha256(),
           "source": "oracle.topk_patterns (Algorithm 2, MNI support by existence search)",
           "M": {}}
    path = os.path.join(HERE, "patterns_rmat18z_top10.json")
    if os.path.exists(path):
        with open(path) as f:
            old = json.load(f)
        if old.get("sha256_graph") == out["sha256_graph"]:
            out["M"] = old["M"]
    for M in Ms:
        t = time.time()
        r = oracle.topk_patterns(g, M, 10)
        out["M"][str(M)] = {"rows": [[x[0], list(x[3]), [list(e) for e in x[2]]] for x in r],
                            "oracle_seconds": time.time() - t}
        print("patterns M", M, time.time() - t, flush=True)
        with open(path, "w") as f:
            json.dump(out, f, separators=(",", ":"))


# ---- vertex-weighted cliques: R-MAT 11 with weights 0..1000, top-100 ----------------------
WCLIQUE_CASE = ("rmat", (11, 16), {"seed": 11}, (0, 1000, 211))


def wclique_graph():
    import synth
    fn, args, kw, (lo, hi, wseed) = WCLIQUE_CASE
    g = getattr(synth, fn)(*args, **kw)
    g.weights = synth.weights_uniform(g.n, lo, hi, seed=wseed)
    return g


def make_wcliques_rmat11(k=100):
    import oracle
    g = wclique_graph()
    t = time.time()
    r = oracle.topk_wcliques(g, k)
    out = {"case": "wcliques_rmat11_top100", "recipe": [WCLIQUE_CASE[0], list(WCLIQUE_CASE[1]),
                                                       WCLIQUE_CASE[2], list(WCLIQUE_CASE[3])],
           "sha256_graph": g.sha256(),
           "source": "oracle.topk_wcliques (Algorithm 1 with the clique functions, vertex-weight "
                     "score, bound w(V) + w(P))",
           "oracle_seconds": time.time() - t,
           "rows": [[x[0], list(x[1])] for x in r]}
    with open(os.path.join(HERE, "wcliques_rmat11_top100.json"), "w") as f:
        json.dump(out, f, separators=(",", ":"))
    print("wcliques", out["oracle_seconds"], flush=True)


CASES = {
    "cliques_er1200": lambda: make_cliques("er1200_p025_s91"),
    "cliques_er1000": lambda: make_cliques("er1000_p033_s5", k_all=300, k_max=100),
    "cliques_chunglu100k": lambda: make_chunglu("chunglu100k"),
    "iso_rmat20": make_iso_rmat20,
    "patterns_rmat18z": make_patterns_rmat18z,
    "wcliques_rmat11": make_wcliques_rmat11,
}

if __name__ == "__main__":
    names = sys.argv[1:] or list(CASES)
    for nm in names:
        CASES[nm]()
