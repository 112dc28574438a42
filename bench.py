"""Benchmark: exact top-k subgraph discovery on one B300 (prints one JSON line).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl nuri|reference]

Default workload (the configuration the headline metric is quoted on): top-100 cliques by
size on a Chung-Lu power-law graph (n = 1M, mean degree 20, exponent 2.1) with 50 planted
cliques of 15..30 vertices, seed 0.  The graph is loaded once and stays resident; a step is one
top-k query (seeds, bucketed frontier rounds, bitmap tail, threshold, top-k merge).  L2 is
flushed (a 256 MB write) before every step; each step is timed with CUDA events on the
query's stream.  Secondary workloads are reported under "workloads".

--impl reference times the CPU oracle (Algorithm 1 as the paper states it) on a bounded
sample of the same workload.  Under torchrun every rank runs its own replica (no data-path
collective exists in this path); rank 0 prints the line.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "expansions/s, time-to-top-k vs plain GPU path; serving p50/p99 latency"


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


def alu_peak_gops():
    """Peak rate of 64-bit bitmap word operations (AND / AND-NOT of an adjacency-row word into
    a candidate mask): 148 SMs x 64 32-bit logical operations per clock per SM / 2 (a 64-bit
    word takes two) x the maximum SM clock (MEASURED_PEAKS.json, else 2032 MHz)."""
    mhz = 2032.0
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            mhz = float(json.load(f).get("sm_max_mhz", mhz))
    except Exception:
        pass
    return 148 * 64 / 2 * mhz * 1e6 / 1e9


class Clocks:
    """Samples nvidia-smi every 200 ms while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.rows = []
        self.proc = None
        self.index = index

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm = [float(r[1]) for r in self.rows if len(r) > 2 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if len(r) > 2 and r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in self.rows:
            for i, nm in enumerate(names):
                if len(r) > 5 + i and r[5 + i].lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(self.rows)}


def source_digest():
    """SHA-256 (16 hex) of the clique engine's source: DRAM counters taken on another
    version of the kernels no longer describe them."""
    import hashlib
    h = hashlib.sha256()
    for f in ("cliques.cu", "nuri_internal.cuh", "topk_common.cuh"):
        with open(os.path.join(ROOT, "paper_1807_08888_b300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def rooflines(total_ms, csr_bytes, csr_ms, csr_launches, tail_words, tail_ms, tail_launches):
    """HBM rooflines of the two clique kernels, dominant (larger share of the step) first,
    then the task kernel's bit-operation rate against a derived ALU peak.

    Algorithmic bytes per unit of work: a CSR expansion reads 4 B per adjacency entry it
    intersects (the kernel counts them, stats adj_bytes); a bitmap-tail node combines 64-bit
    row words into candidate masks, 8 B per word (stats tail_words).  achieved = those bytes
    per launch / the launch's CUDA-event time; traffic = DRAM bytes per launch, from the ncu
    capture in profiles/traffic.json (DRAM bytes per algorithmic byte on the 200k-vertex case,
    times this launch's algorithmic bytes), or null when the kernels changed since."""
    peak, peak_kind = peaks()
    traffic = {}
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            traffic = json.load(f)
    except Exception:
        pass
    digest = source_digest()

    def line(kernel, key, alg_bytes, ms, launches):
        ms = max(ms, 1e-9)
        per_launch = alg_bytes / max(launches, 1)
        achieved = alg_bytes / (ms / 1e3) / 1e9
        t = traffic.get(key) or {}
        tr = (t["dram_per_algorithmic_byte"] * per_launch
              if t.get("source_digest") == digest and t.get("dram_per_algorithmic_byte")
              else None)
        return {"bound": "hbm", "kernel": kernel, "achieved": achieved, "peak": peak,
                "unit": "GB/s", "frac": achieved / peak,
                "peak_source": f"{peak_kind} hbm_gbs (MEASURED_PEAKS.json), of {peak_kind}",
                "traffic": tr, "algorithmic_bytes_per_launch": per_launch,
                "avg_launch_ms": ms / max(launches, 1), "launches": launches,
                "share_of_step": ms / total_ms,
                "traffic_source": t.get("source") if tr is not None else
                "no capture of this kernel version"}

    csr = line("k_clique_expand", "k_clique_expand", csr_bytes, csr_ms, csr_launches)
    tail = line("k_clique_tasks", "k_clique_tasks", 8.0 * tail_words, tail_ms, tail_launches)
    apeak = alu_peak_gops()
    tach = (tail_words / (tail_ms / 1e3)) / 1e9 if tail_ms > 0 else 0.0
    alu = {"bound": "alu", "kernel": "k_clique_tasks", "achieved": tach, "peak": apeak,
           "unit": "Gword-ops/s", "frac": tach / apeak,
           "peak_source": "derived: 148 SMs x 32 64-bit logical ops/clk x sm_max_mhz"}
    return (csr, tail, alu) if csr_ms >= tail_ms else (tail, csr, alu)


def combine_ranks(total_ms, total_units, dist=None, device="cpu"):
    """Whole-job aggregate over replicas: the slowest rank's time and the units of all ranks
    (value = units / time).  Works with any torch.distributed backend (gloo on CPU in tests,
    NCCL on the GPUs)."""
    if dist is None:
        return float(total_ms), float(total_units)
    import torch
    tm = torch.tensor([float(total_ms)], dtype=torch.float64, device=device)
    tu = torch.tensor([float(total_units)], dtype=torch.float64, device=device)
    dist.all_reduce(tm, op=dist.ReduceOp.MAX)
    dist.all_reduce(tu, op=dist.ReduceOp.SUM)
    return float(tm.item()), float(tu.item())


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def cpu_baseline(budget_expansions=30_000_000):
    """The oracle (Algorithm 1, paper order and priorities) on a bounded sample: the first
    `budget` expansions of the headline workload, single thread."""
    import oracle
    import synth
    g = synth.workload("chunglu1m")
    t = time.perf_counter()
    r = oracle.topk_cliques(g, 100, budget=budget_expansions)
    wall = time.perf_counter() - t
    out = {"value": r.expansions / r.seconds if r.seconds > 0 else None,
           "unit": "expansions/s", "cores": 1, "kind": "oracle",
           "sample": f"first {r.expansions} expansions of top-100 cliques on chunglu1m "
                     f"(budget {budget_expansions}; complete={r.complete}), "
                     f"{r.seconds:.1f} s inside the oracle, {wall:.1f} s with graph build"}
    # like for like where the oracle finishes: its time to the top-k on the ER workload
    # (the GPU figure for the same query is workloads.er2000_top10_cliques)
    ge = synth.workload("er2000")
    re_ = oracle.topk_cliques(ge, 10)
    out["er2000_top10_time_to_topk_ms"] = re_.seconds * 1e3
    out["er2000_top10_complete"] = bool(re_.complete)
    return out


def run_reference(args, world, rank):
    if rank != 0:
        return
    vals, walls = [], []
    base = None
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        b = cpu_baseline(budget_expansions=args.ref_budget)
        if i >= args.warmup:
            vals.append(b["value"])
            walls.append(time.perf_counter() - t0)
            base = b
    v = float(np.mean(vals))
    line = {"metric": METRIC, "value": v, "unit": "expansions/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * float(np.mean(walls)),  # one bounded oracle sample a step
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
            "data": "synthetic (seeded Chung-Lu + planted cliques)", "impl": "reference",
            "config": {"workload": "chunglu1m_top100_cliques", "n": 1_000_000, "k": 100},
            "cpu_baseline": dict(base, value=v),
            "e2e": {"value": v, "unit": "expansions/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="nuri", choices=["nuri", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra", action="store_true")
    ap.add_argument("--ref-budget", type=int, default=30_000_000)
    ap.add_argument("--workload", default="headline",
                    choices=["headline", "serving", "profile-clique", "profile-clique1m",
                             "profile-iso", "profile-iso-edge", "profile-wcliques",
                             "profile-esu", "profile-hop", "profile-patterns"])
    ap.add_argument("--repeat", type=int, default=1,
                    help="profile cases: queries run one after another on the loaded graph")
    ap.add_argument("--serving-graph", default="rmat22")
    ap.add_argument("--requests", type=int, default=1000)
    ap.add_argument("--calibrate", type=int, default=200)
    ap.add_argument("--slots", type=int, default=8)
    ap.add_argument("--request-budget-ms", type=float, default=60000.0)
    ap.add_argument("--serving-kinds", default="mix", choices=["mix", "iso", "clique"],
                    help="serving: the 50/50 stream, or only its isomorphism or clique requests "
                         "(thinned from a stream at twice the rate, so each kind keeps its "
                         "arrival process)")
    args = ap.parse_args()
    world, rank, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, world, rank)
        return

    import torch
    import paper_1807_08888_b300 as nuri
    import synth

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    stream = torch.cuda.current_stream()
    sptr = stream.cuda_stream
    if args.workload.startswith("profile-"):
        profile_case(args.workload[len("profile-"):], nuri, sptr, args.repeat)
        return
    if args.workload == "serving":
        res = serving(args, nuri, torch, sptr)
        line = {"metric": METRIC, "workload": "serving", "unit": "ms", "n_gpus": world,
                "higher_is_better": False, "data": "synthetic (seeded R-MAT + Poisson arrivals)",
                "dtype": "int32", "serving": res}
        if rank == 0:
            print(json.dumps(line), flush=True)
        return
    g = synth.workload("chunglu1m")
    G = nuri.load_graph(g.n, g.src, g.dst, stream=sptr)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.int32, device="cuda")
    k = 100
    # autotune the dense search's task granularity on this graph (outside the timed region)
    tuned, tuned_ms = nuri.tune_cliques(G, k, stream=sptr)

    def step():
        flush.fill_(1)  # 256 MB write: evicts L2 between steps (outside the timed region)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        r = nuri.topk_cliques(G, k, stream=sptr)
        e1.record(stream)
        torch.cuda.synchronize()
        return r, e0.elapsed_time(e1)

    for _ in range(args.warmup):
        step()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    times, exps, exp_ms, exp_bytes, launches, exp_launches = [], [], [], [], 0, 0
    tail_ms, tail_words, tail_launches = 0.0, 0, 0
    with Clocks(local) as clk:
        for _ in range(args.steps):
            r, ms = step()
            times.append(ms)
            exps.append(r.stats["expansions"])
            exp_ms.append(r.stats["expand_ms"])
            exp_bytes.append(r.stats["adj_bytes"])
            launches += r.stats["launches"]
            exp_launches += r.stats["expand_launches"]
            tail_ms += r.stats["tail_ms"]
            tail_words += r.stats["tail_words"]
            tail_launches += r.stats["tail_launches"]
    torch.cuda.synchronize()
    total_ms = float(sum(times))
    total_exp = float(sum(exps))
    if dist:
        total_ms, total_exp = combine_ranks(total_ms, total_exp, dist, device="cuda")
    value = total_exp / (total_ms / 1e3)
    roofs = rooflines(total_ms, sum(exp_bytes), sum(exp_ms), exp_launches,
                      tail_words, tail_ms, tail_launches)
    dominant, secondary = roofs[0], roofs[1]
    last = r
    line = {
        "metric": METRIC, "value": value, "unit": "expansions/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
        "data": "synthetic (seeded Chung-Lu power-law graph + 50 planted cliques)",
        "config": {"workload": "chunglu1m_top100_cliques", "n": g.n, "m_input": g.m, "k": k,
                   "l2": "flushed (256 MB write) before every step",
                   "autotune": {"task_split_above": tuned, "tuning_query_ms": tuned_ms,
                                "candidates": [48, 96, 128, 192],
                                "e2e": "fresh graph each step: default 96"},
                   "parallelism":
                   "replicas" if world > 1 else "single GPU"},
        "time_to_topk_ms": total_ms / args.steps,
        "expansions_per_step": total_exp / args.steps / world,
        "threshold": last.stats["threshold"], "rounds_per_step": last.stats["rounds"],
        "gpu_launches": launches, "gpu_launches_per_step": launches / args.steps,
        "roofline": dominant, "roofline_secondary": secondary, "roofline_alu": roofs[2],
        "clocks": clk.summary(),
    }
    # end to end through the public API with host buffers: H2D of the edge list, graph build,
    # query, D2H of the result rows, every step
    pin_s = torch.from_numpy(g.src).pin_memory()
    pin_d = torch.from_numpy(g.dst).pin_memory()
    e2e_t, e2e_exp, d2h = [], [], 0
    e2e_steps = min(args.steps, 2)
    for i in range(1 + e2e_steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        G2 = nuri.load_graph(g.n, pin_s.numpy(), pin_d.numpy(), stream=sptr)
        r2 = nuri.topk_cliques(G2, k, stream=sptr)
        G2.free()
        t1 = time.perf_counter()
        if i >= 1:
            e2e_t.append(t1 - t0)
            e2e_exp.append(r2.stats["expansions"])
            d2h = sum(8 + 4 * len(x[1]) for x in r2)
    line["e2e"] = {"value": sum(e2e_exp) / sum(e2e_t), "unit": "expansions/s",
                   "ms_per_step": 1e3 * sum(e2e_t) / len(e2e_t),
                   "h2d_bytes_per_step": int(pin_s.numel() * 4 * 2),
                   "d2h_bytes_per_step": int(d2h),
                   "includes": "H2D edge list, device CSR build, query, D2H rows"}
    if not args.no_extra and rank == 0:
        line["workloads"] = extra_workloads(nuri, torch, sptr, G, g)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args.ref_budget)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def _ms(r):
    return r.stats["device_ms"]


def profile_case(which, nuri, sptr, repeat=1):
    """Cases of each kernel family for ncu captures.  clique1m is the headline query (its graph
    and buffers are about 2 GB; only single-pass metrics are taken on it); clique (200k
    vertices), iso (R-MAT 18), hop and patterns hold a few hundred MB.  `repeat` runs the
    query that many times on the loaded graph (a later query sees warm buffers and local
    memory already set up, as the benchmark's timed steps do)."""
    import synth
    if which in ("clique1m", "clique"):
        g = (synth.workload("chunglu1m") if which == "clique1m"
             else synth.chung_lu_planted(200000, 20.0, 2.1, 20, 15, 30, seed=0))
        G = nuri.load_graph(g.n, g.src, g.dst, stream=sptr)
        for i in range(repeat):
            r = nuri.topk_cliques(G, 100, stream=sptr)
            print(json.dumps({"case": which, "query": i, "stats": r.stats}))
    elif which == "iso":
        g = synth.rmat(18, 16, seed=3)
        g.labels = synth.labels_uniform(g.n, 8, seed=4)
        g.weights = synth.weights_uniform(g.n, 0, 1000, seed=5)
        G = nuri.load_graph(g.n, g.src, g.dst, labels=g.labels, weights=g.weights,
                            index_hops=4, stream=sptr)
        for i in range(repeat):
            r = nuri.topk_iso_batch(G, synth.query_batch(64, seed=1), [1000] * 64, stream=sptr)
            print(json.dumps({"case": which, "query": i, "stats": r[0].stats}))
    elif which == "iso-edge":
        g = synth.rmat(18, 16, seed=3)
        g.labels = synth.labels_uniform(g.n, 8, seed=4)
        g.weights = synth.weights_uniform(g.n, 0, 1000, seed=5)
        g.edge_weights = synth.edge_weights_uniform(g.m, 0, 1000, seed=6)
        G = nuri.load_graph(g.n, g.src, g.dst, labels=g.labels, weights=g.weights,
                            stream=sptr)
        G.set_edge_weights(g.src, g.dst, g.edge_weights, stream=sptr)
        for i in range(repeat):
            r = nuri.topk_iso_batch(G, synth.query_batch(16, seed=1), [100] * 16,
                                    edge_rank=True, stream=sptr)
            print(json.dumps({"case": which, "query": i, "stats": r[0].stats}))
    elif which == "wcliques":
        g = synth.chung_lu_planted(200000, 20.0, 2.1, 20, 15, 30, seed=0)
        w = synth.weights_uniform(g.n, 0, 1000, seed=11)
        G = nuri.load_graph(g.n, g.src, g.dst, weights=w, stream=sptr)
        for i in range(repeat):
            r = nuri.topk_cliques(G, 100, weighted=True, stream=sptr)
            print(json.dumps({"case": which, "query": i, "stats": r.stats}))
    elif which == "esu":
        g = synth.rmat(12, 16, seed=41)
        g.labels = synth.labels_zipf(g.n, 8, 1.2, seed=41)
        G = nuri.load_graph(g.n, g.src, g.dst, labels=g.labels, stream=sptr)
        for i in range(repeat):
            r = nuri.topk_patterns(G, 2, 10, edge_oriented=True, stream=sptr)
            print(json.dumps({"case": which, "query": i, "stats": r.stats}))
    elif which == "hop":
        g = synth.workload("rmat20")
        G = nuri.load_graph(g.n, g.src, g.dst, labels=g.labels, weights=g.weights,
                            index_hops=4, stream=sptr)
        print(json.dumps({"case": which, "info": G.info()}))
    elif which == "patterns":
        g = synth.workload("rmat18z")
        G = nuri.load_graph(g.n, g.src, g.dst, labels=g.labels, stream=sptr)
        r = nuri.topk_patterns(G, 3, 10, stream=sptr)
        print(json.dumps({"case": which, "stats": r.stats}))


def _pct(v, q):
    """The q-quantile of the latencies v (nearest rank), None when there are none."""
    if not v:
        return None
    v = sorted(v)
    return v[min(len(v) - 1, int(q * len(v)))]


def serving(args, nuri, torch, sptr):
    """Open-loop serving on the resident R-MAT scale-22 graph: Poisson arrivals of a 50/50 mix
    of top-k clique (k 1..100) and isomorphism (3..8 vertices, k 10..1000) requests at 0.5, 1
    and 2 times the plain one-at-a-time throughput mu1 (calibrated on 200 requests)."""
    import synth
    g = synth.workload(args.serving_graph)
    t0 = time.perf_counter()
    G = nuri.load_graph(g.n, g.src, g.dst, labels=g.labels, weights=g.weights, index_hops=4,
                        stream=sptr)
    load_s = time.perf_counter() - t0
    nuri.set_time_budget(args.request_budget_ms)

    def run_alone(r):
        if r["kind"] == "clique":
            return nuri.topk_cliques(G, r["k"], stream=sptr)
        return nuri.topk_iso(G, r["query"], r["k"], stream=sptr)

    kinds = args.serving_kinds

    def stream(count, rate, seed):
        if kinds == "mix":
            return synth.serving_requests(count, rate=rate, seed=seed)
        both = synth.serving_requests(2 * count + 256, rate=2 * rate, seed=seed)
        return [r for r in both if r["kind"] == kinds][:count]

    calib = stream(args.calibrate, 1.0, 100)
    for r in calib[:5]:  # warm-up (a request may hit the per-request time budget)
        try:
            run_alone(r)
        except nuri.NuriError:
            pass
    t0 = time.perf_counter()
    fails = 0
    for r in calib:
        try:
            run_alone(r)
        except nuri.NuriError:
            fails += 1
    mu1 = len(calib) / (time.perf_counter() - t0)
    out = {"graph": args.serving_graph, "edges": G.info()["num_edges"], "load_s": load_s,
           "mu1_req_per_s": mu1, "calibration_failures": fails, "slots": args.slots,
           "requests_per_rate": args.requests, "kinds": kinds, "rates": {}}
    for i, f in enumerate((0.5, 1.0, 2.0)):
        rate = f * mu1
        reqs = stream(args.requests, rate, i)
        srv = nuri.Server(G, slots=args.slots, max_batch=64)
        tickets = [None] * len(reqs)
        start = time.perf_counter()

        def submitter():
            for j, r in enumerate(reqs):
                delay = start + r["t"] - time.perf_counter()
                if delay > 0:
                    time.sleep(delay)
                tickets[j] = (srv.submit_cliques(r["k"]) if r["kind"] == "clique"
                              else srv.submit_iso(r["query"], r["k"]))

        th = threading.Thread(target=submitter)
        th.start()
        lat, errs, done = [], 0, 0
        by_kind = {"clique": [], "iso": []}
        pending = set()
        j = 0
        while done < len(reqs):
            while j < len(reqs) and tickets[j] is not None:
                pending.add(j)
                j += 1
            finished = []
            for q in pending:
                try:
                    rr = srv.poll(tickets[q])
                except nuri.NuriError:
                    rr = ("error", None)
                if rr is None:
                    continue
                finished.append(q)
                if rr[0] == "error":
                    errs += 1
                else:
                    # latency from the scheduled arrival (includes any submission delay)
                    lat.append((time.perf_counter() - start - reqs[q]["t"]) * 1e3)
                    by_kind[reqs[q]["kind"]].append(lat[-1])
            for q in finished:
                pending.discard(q)
            done += len(finished)
            if not finished:
                time.sleep(0.0005)
        wall = time.perf_counter() - start
        th.join()
        st = srv.stats()
        srv.close()
        lat.sort()
        out["rates"][f"{f}x"] = {
            "offered_req_per_s": rate, "completed_req_per_s": len(reqs) / wall,
            "p50_ms": lat[len(lat) // 2] if lat else None,
            "p99_ms": lat[min(len(lat) - 1, int(0.99 * len(lat)))] if lat else None,
            "errors": errs, "iso_batches": st["iso_batches"],
            "iso_requests": st["iso_batched_requests"],
            "by_kind": {kd: {"count": len(v), "p50_ms": _pct(v, 0.5), "p99_ms": _pct(v, 0.99),
                             "max_ms": max(v) if v else None}
                        for kd, v in by_kind.items()}}
    nuri.set_time_budget(0)
    return out


def clique_batch_vs_plain(nuri, torch, G, sptr, count=16, seed=5):
    """Top-k clique requests (k uniform 1..100) on one graph: one nuri_topk_batch call (one
    shared search for the largest k) against the plain path (one nuri_topk_cliques call per
    request), each timed with CUDA events on the query stream."""
    rng = np.random.default_rng(seed)
    ks = [int(x) for x in rng.integers(1, 101, size=count)]
    stream = torch.cuda.current_stream()

    def timed(fn):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        r = fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return r, e0.elapsed_time(e1)

    timed(lambda: nuri.topk_batch(G, [("clique", k) for k in ks], stream=sptr))  # warm-up
    batch, bms = timed(lambda: nuri.topk_batch(G, [("clique", k) for k in ks], stream=sptr))
    plain_ms, plain_exp, same = 0.0, 0, True
    for k, b in zip(ks, batch):
        r, ms = timed(lambda: nuri.topk_cliques(G, k, stream=sptr))
        plain_ms += ms
        plain_exp += r.stats["expansions"]
        same &= [tuple(x) for x in r] == [tuple(x) for x in b]
    return {"requests": count, "ks": ks, "batched_time_to_topk_ms": bms,
            "plain_time_to_topk_ms": plain_ms, "batched_speedup": plain_ms / bms,
            "batched_expansions": batch[0].stats["expansions"], "plain_expansions": plain_exp,
            "batched_expansions_per_s": batch[0].stats["expansions"] / (bms / 1e3),
            "plain_expansions_per_s": plain_exp / (plain_ms / 1e3),
            "rows_equal_plain": bool(same)}


def weighted_rankings(nuri, sptr, g_headline):
    """The weighted rankings: top-100 cliques by vertex weight on the headline graph with
    weights uniform 0..1000, and 16 isomorphism queries of the R-MAT 20 workload at top-100
    ranked by edge weight (edge weights uniform 0..1000) next to the same queries ranked by
    vertex weight.  Device time of the query (CUDA events inside the library), algorithmic
    bytes from the kernels' counters over that time against the measured copy bandwidth."""
    import synth
    hbm = peaks()[0]
    out = {}
    if g_headline is not None:
        w = synth.weights_uniform(g_headline.n, 0, 1000, seed=11)
        G = nuri.load_graph(g_headline.n, g_headline.src, g_headline.dst, weights=w, stream=sptr)
        nuri.topk_cliques(G, 100, weighted=True, stream=sptr)  # warm-up
        r = nuri.topk_cliques(G, 100, weighted=True, stream=sptr)
        ms = _ms(r)
        out["chunglu1m_top100_weighted_cliques"] = {
            "time_to_topk_ms": ms, "expansions": r.stats["expansions"],
            "expansions_per_s": r.stats["expansions"] / (ms / 1e3),
            "algorithmic_gbs": r.stats["adj_bytes"] / (ms / 1e3) / 1e9,
            "hbm_frac_of_measured": r.stats["adj_bytes"] / (ms / 1e3) / 1e9 / hbm,
            "top_score": r[0][0] if r else None, "launches": r.stats["launches"]}
        G.free()
    g = synth.workload("rmat20")
    g.edge_weights = synth.edge_weights_uniform(g.m, 0, 1000, seed=12)
    G = nuri.load_graph(g.n, g.src, g.dst, labels=g.labels, weights=g.weights, index_hops=4,
                        stream=sptr)
    G.set_edge_weights(g.src, g.dst, g.edge_weights, stream=sptr)
    qs = synth.query_batch(64, seed=1)[:16]
    res = {}
    for name, edge in (("edge_weight", True), ("vertex_weight", False)):
        nuri.topk_iso_batch(G, qs, [100] * 16, edge_rank=edge, stream=sptr)  # warm-up
        rb = nuri.topk_iso_batch(G, qs, [100] * 16, edge_rank=edge, stream=sptr)
        ms = _ms(rb[0])
        res[name] = {"time_to_topk_ms": ms, "expansions": rb[0].stats["expansions"],
                     "expansions_per_s": rb[0].stats["expansions"] / (ms / 1e3),
                     "algorithmic_gbs": rb[0].stats["adj_bytes"] / (ms / 1e3) / 1e9,
                     "hbm_frac_of_measured": rb[0].stats["adj_bytes"] / (ms / 1e3) / 1e9 / hbm}
    out["rmat20_iso16_top100_by_edge_weight"] = res
    G.free()
    return out


def extra_workloads(nuri, torch, sptr, G_headline=None, g_headline=None):
    """The other configurations: clique requests batched vs one at a time on the headline
    graph, ER planted clique, the 64-query isomorphism batch (batched launch vs one query at a
    time), pattern mining M = 1..5, the weighted rankings, and the pruning gain of Algorithm 2
    over exhaustive edge-oriented expansion."""
    import synth
    out = {}
    if G_headline is not None:
        out["chunglu1m_clique_batch16"] = clique_batch_vs_plain(nuri, torch, G_headline, sptr)
    out.update(weighted_rankings(nuri, sptr, g_headline))
    g = synth.workload("er2000")
    G = nuri.load_graph(g.n, g.src, g.dst, stream=sptr)
    for _ in range(3):
        nuri.topk_cliques(G, 10, stream=sptr)
    r = nuri.topk_cliques(G, 10, stream=sptr)
    out["er2000_top10_cliques"] = {"time_to_topk_ms": _ms(r), "expansions": r.stats["expansions"],
                                   "expansions_per_s": r.stats["expansions"] / (_ms(r) / 1e3)}
    G.free()

    g = synth.workload("rmat20")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    G = nuri.load_graph(g.n, g.src, g.dst, labels=g.labels, weights=g.weights, index_hops=4,
                        stream=sptr)
    load_s = time.perf_counter() - t0
    qs = synth.query_batch(64, seed=1)
    ks = [1000] * 64
    nuri.topk_iso_batch(G, qs, ks, stream=sptr)  # warm-up
    bt = []
    for _ in range(3):
        rb = nuri.topk_iso_batch(G, qs, ks, stream=sptr)
        bt.append(_ms(rb[0]))
    exp_b = rb[0].stats["expansions"]
    plain_ms, exp_p = 0.0, 0
    for q in qs:
        rp = nuri.topk_iso(G, q, 1000, stream=sptr)
        plain_ms += _ms(rp)
        exp_p += rp.stats["expansions"]
    bms = float(np.median(bt))
    out["rmat20_iso64_top1000"] = {
        "batched_time_to_topk_ms": bms, "plain_time_to_topk_ms": plain_ms,
        "batched_expansions_per_s": exp_b / (bms / 1e3),
        "plain_expansions_per_s": exp_p / (plain_ms / 1e3),
        "batched_speedup": plain_ms / bms, "expansions_batched": exp_b,
        "expansions_plain": exp_p, "graph_load_and_index_s": load_s,
        "edges": G.info()["num_edges"]}
    G.free()

    g = synth.workload("rmat18z")
    G = nuri.load_graph(g.n, g.src, g.dst, labels=g.labels, stream=sptr)
    pm = {}
    for M in (1, 2, 3, 4, 5):
        nuri.topk_patterns(G, M, 10, stream=sptr)
        r = nuri.topk_patterns(G, M, 10, stream=sptr)
        pm[f"M{M}"] = {"time_to_topk_ms": _ms(r), "top_support": r[0][0] if r else None,
                       "kth_support": r[-1][0] if r else None, "candidates": r.stats["expansions"]}
    out["rmat18z_top10_patterns"] = pm
    G.free()

    # the pruning gain: Algorithm 2 against exhaustive edge-oriented expansion (every
    # connected M-edge subgraph grown and grouped, no pruning), same rows
    g = synth.rmat(12, 16, seed=41)
    g.labels = synth.labels_zipf(g.n, 8, 1.2, seed=41)
    G = nuri.load_graph(g.n, g.src, g.dst, labels=g.labels, stream=sptr)
    gain = {}
    for M in (1, 2, 3):
        nuri.topk_patterns(G, M, 10, stream=sptr)
        a = nuri.topk_patterns(G, M, 10, stream=sptr)
        e = nuri.topk_patterns(G, M, 10, edge_oriented=True, stream=sptr)
        gain[f"M{M}"] = {
            "algorithm2_ms": _ms(a), "algorithm2_candidates": a.stats["expansions"],
            "edge_oriented_ms": _ms(e), "edge_oriented_subgraphs": e.stats["expansions"],
            "embeddings": e.stats["results_stored"], "patterns": e.stats["dequeued"],
            "same_rows": [tuple(x) for x in a] == [tuple(x) for x in e]}
    out["rmat12z_top10_patterns_pruning_gain"] = gain
    G.free()
    return out


if __name__ == "__main__":
    main()
