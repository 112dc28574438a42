// C ABI of libnuri (declared in include/nuri.h): argument checks, error conversion, result
// allocation.  Every entry point catches the library's internal errors and returns a status.
#include <atomic>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <algorithm>
#include <mutex>
#include <new>
#include <utility>
#include <vector>

#include "nuri_internal.cuh"

namespace nuri {

// patterns_edge.cu: top-k patterns by exhaustive edge-oriented expansion
void topk_patterns_edge(nuri_graph* g, int32_t M, int32_t k, uint32_t flags, cudaStream_t s,
                        nuri_result** out);

static thread_local char g_err[1024] = "";

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

const char* last_error() { return g_err; }

static std::atomic<uint64_t> g_budget_ns{0};
std::atomic<int> g_cuda_site{0};
uint64_t time_budget_ns() { return g_budget_ns.load(); }

__global__ void k_set_deadline(uint64_t* deadline, uint64_t budget_ns) {
  if (threadIdx.x == 0 && blockIdx.x == 0)
    *deadline = budget_ns ? global_ns() + budget_ns : ~0ull;
}

// One pool per device, created on first use.  Its release threshold keeps up to
// NURI_POOL_KEEP_MB (default 8192) MB of freed memory cached between synchronisations.
cudaMemPool_t device_pool() {
  static std::mutex mu;
  static std::vector<cudaMemPool_t> pools;
  int dev = 0;
  NURI_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(mu);
  if ((int)pools.size() <= dev) pools.resize(dev + 1, nullptr);
  if (!pools[dev]) {
    cudaMemPoolProps props;
    memset(&props, 0, sizeof(props));
    props.allocType = cudaMemAllocationTypePinned;
    props.handleTypes = cudaMemHandleTypeNone;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t pool;
    NURI_CUDA(cudaMemPoolCreate(&pool, &props));
    uint64_t keep = 8192ull << 20;
    if (const char* e = getenv("NURI_POOL_KEEP_MB")) keep = (uint64_t)atoll(e) << 20;
    NURI_CUDA(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep));
    pools[dev] = pool;
  }
  return pools[dev];
}

nuri_result* new_result(int kind, int32_t count, int64_t nverts, int64_t nedges, bool labels) {
  nuri_result* r = (nuri_result*)calloc(1, sizeof(nuri_result));
  if (!r) NURI_FAIL(NURI_ERR_OOM, "host allocation failed");
  r->count = count;
  r->kind = kind;
  r->score = (int64_t*)calloc((size_t)count + 1, sizeof(int64_t));
  r->vert_off = (int32_t*)calloc((size_t)count + 1, sizeof(int32_t));
  r->edge_off = (int32_t*)calloc((size_t)count + 1, sizeof(int32_t));
  r->verts = (int32_t*)calloc((size_t)nverts + 1, sizeof(int32_t));
  r->edges = (int32_t*)calloc((size_t)(2 * nedges) + 2, sizeof(int32_t));
  r->labels = labels ? (int32_t*)calloc((size_t)nverts + 1, sizeof(int32_t)) : nullptr;
  if (!r->score || !r->vert_off || !r->edge_off || !r->verts || !r->edges ||
      (labels && !r->labels)) {
    nuri_free_result(r);
    NURI_FAIL(NURI_ERR_OOM, "host allocation failed");
  }
  return r;
}

template <class F>
static nuri_status guarded(F&& f) {
  g_err[0] = 0;
  try {
    f();
    return NURI_OK;
  } catch (const Err& e) {
    return e.code;
  } catch (const std::bad_alloc&) {
    set_error("host allocation failed");
    return NURI_ERR_OOM;
  } catch (...) {
    set_error("unexpected internal error");
    return NURI_ERR_CUDA;
  }
}

}  // namespace nuri

using namespace nuri;

extern "C" {

const char* nuri_last_error(void) { return nuri::last_error(); }

const char* nuri_version(void) { return "nuri-b300 0.1 (sm_103a)"; }

nuri_status nuri_load_graph(int32_t n, int64_t m, const int32_t* src, const int32_t* dst,
                            const uint8_t* labels, const int32_t* weights, int32_t index_hops,
                            uint32_t flags, void* stream, nuri_graph** out) {
  return guarded([&] {
    if (!out) NURI_FAIL(NURI_ERR_INVALID, "nuri_load_graph: out is NULL");
    *out = nullptr;
    if (n < 0 || m < 0) NURI_FAIL(NURI_ERR_INVALID, "nuri_load_graph: negative size");
    if (m > 0 && (!src || !dst)) NURI_FAIL(NURI_ERR_INVALID, "nuri_load_graph: NULL edge arrays");
    if (index_hops < 0 || index_hops > 7)
      NURI_FAIL(NURI_ERR_INVALID, "nuri_load_graph: index_hops must be in 0..7");
    cudaStream_t s = (cudaStream_t)stream;
    nuri_graph* g = new nuri_graph();
    g->stream = s;
    try {
      build_graph(g, n, m, src, dst, labels, weights, index_hops, flags, s);
    } catch (...) {
      delete g;
      throw;
    }
    *out = g;
  });
}

void nuri_free_graph(nuri_graph* g) {
  if (!g) return;
  cudaStream_t s = g->stream;
  delete g;  // DBuf destructors free stream-ordered
  cudaStreamSynchronize(s);
}

nuri_status nuri_set_edge_weights(nuri_graph* g, int64_t m, const int32_t* src,
                                  const int32_t* dst, const int32_t* w, uint32_t flags,
                                  void* stream) {
  return guarded([&] {
    if (!g) NURI_FAIL(NURI_ERR_INVALID, "nuri_set_edge_weights: NULL graph");
    if (m < 0) NURI_FAIL(NURI_ERR_INVALID, "nuri_set_edge_weights: negative size");
    if (m > 0 && (!src || !dst || !w))
      NURI_FAIL(NURI_ERR_INVALID, "nuri_set_edge_weights: NULL arrays");
    set_edge_weights(g, m, src, dst, w, (flags & NURI_LOAD_DEVICE_INPUT) != 0,
                     (cudaStream_t)stream);
  });
}

nuri_status nuri_graph_get_info(const nuri_graph* g, nuri_graph_info* info) {
  return guarded([&] {
    if (!g || !info) NURI_FAIL(NURI_ERR_INVALID, "nuri_graph_get_info: NULL argument");
    memset(info, 0, sizeof(*info));
    info->n = g->d.n;
    info->num_labels = g->d.L;
    info->num_edges = g->num_edges;
    info->dropped = g->dropped;
    info->max_degree = g->d.max_deg;
    info->max_out_degree = g->d.max_out;
    info->index_hops = g->d.H;
    info->device_bytes = g->device_bytes();
  });
}

nuri_status nuri_tune_cliques(nuri_graph* g, int32_t k, uint32_t flags, void* stream,
                              int32_t* chosen, double* best_ms) {
  return guarded([&] {
    if (!g) NURI_FAIL(NURI_ERR_INVALID, "nuri_tune_cliques: NULL graph");
    if (k < 1) NURI_FAIL(NURI_ERR_INVALID, "nuri_tune_cliques: k must be >= 1");
    // candidate task granularities of the dense-record search (node size above which a
    // node's children become tasks); each is timed on one query, the fastest is kept
    static const int32_t cand[] = {48, 96, 128, 192};
    int32_t best = 0;
    double best_t = 0.0;
    const int32_t before = g->clique_split_bits;
    for (int32_t c : cand) {
      g->clique_split_bits = c;
      nuri_result* r = nullptr;
      try {
        topk_cliques(g, k, flags, 0, (cudaStream_t)stream, &r);
      } catch (...) {
        g->clique_split_bits = before;
        throw;
      }
      const double t = r->stats.device_ms;
      nuri_free_result(r);
      if (best == 0 || t < best_t) {
        best = c;
        best_t = t;
      }
    }
    g->clique_split_bits = best;
    if (chosen) *chosen = best;
    if (best_ms) *best_ms = best_t;
  });
}

nuri_status nuri_topk_cliques(nuri_graph* g, int32_t k, int32_t rank, uint32_t flags,
                              int64_t frontier_cap, void* stream, nuri_result** out) {
  return guarded([&] {
    if (!g || !out) NURI_FAIL(NURI_ERR_INVALID, "nuri_topk_cliques: NULL argument");
    *out = nullptr;
    if (k < 1) NURI_FAIL(NURI_ERR_INVALID, "nuri_topk_cliques: k must be >= 1");
    if (rank != NURI_RANK_SIZE && rank != NURI_RANK_WEIGHT_SUM)
      NURI_FAIL(NURI_ERR_INVALID, "nuri_topk_cliques: rank must be NURI_RANK_SIZE or WEIGHT_SUM");
    if (frontier_cap < 0) NURI_FAIL(NURI_ERR_INVALID, "nuri_topk_cliques: negative frontier_cap");
    if (rank == NURI_RANK_WEIGHT_SUM) {
      if (!g->d.weights) NURI_FAIL(NURI_ERR_INVALID, "nuri_topk_cliques: graph has no weights");
      topk_wcliques(g, k, flags, (cudaStream_t)stream, out);
    } else {
      topk_cliques(g, k, flags, frontier_cap, (cudaStream_t)stream, out);
    }
  });
}

nuri_status nuri_topk_iso(nuri_graph* g, const nuri_query* q, int32_t k, int32_t rank,
                          uint32_t flags, void* stream, nuri_result** out) {
  return nuri_topk_iso_batch(g, 1, q, &k, rank, flags, stream, out);
}

nuri_status nuri_topk_iso_batch(nuri_graph* g, int32_t nqueries, const nuri_query* qs,
                                const int32_t* ks, int32_t rank, uint32_t flags, void* stream,
                                nuri_result** outs) {
  return guarded([&] {
    if (!g || !qs || !ks || !outs) NURI_FAIL(NURI_ERR_INVALID, "nuri_topk_iso: NULL argument");
    if (nqueries < 1) NURI_FAIL(NURI_ERR_INVALID, "nuri_topk_iso: no queries");
    for (int i = 0; i < nqueries; ++i) outs[i] = nullptr;
    if (rank != NURI_RANK_WEIGHT_SUM && rank != NURI_RANK_DEGREE_SUM &&
        rank != NURI_RANK_EDGE_WEIGHT_SUM)
      NURI_FAIL(NURI_ERR_INVALID,
                "nuri_topk_iso: rank must be WEIGHT_SUM, DEGREE_SUM or EDGE_WEIGHT_SUM");
    if (!g->d.labels || !g->d.lsoff) NURI_FAIL(NURI_ERR_INVALID, "nuri_topk_iso: graph has no labels");
    if (rank == NURI_RANK_WEIGHT_SUM && !g->d.weights)
      NURI_FAIL(NURI_ERR_INVALID, "nuri_topk_iso: graph has no weights");
    if (rank == NURI_RANK_EDGE_WEIGHT_SUM && !g->d.ew)
      NURI_FAIL(NURI_ERR_INVALID, "nuri_topk_iso: graph has no edge weights");
    for (int i = 0; i < nqueries; ++i) {
      if (ks[i] < 1) NURI_FAIL(NURI_ERR_INVALID, "nuri_topk_iso: k must be >= 1");
      const nuri_query& q = qs[i];
      if (q.nq < 1 || q.nq > 8) NURI_FAIL(NURI_ERR_INVALID, "nuri_topk_iso: query size must be 1..8");
      if (q.ne < 0 || (q.ne > 0 && (!q.src || !q.dst)) || !q.labels)
        NURI_FAIL(NURI_ERR_INVALID, "nuri_topk_iso: bad query arrays");
    }
    topk_iso_batch(g, nqueries, qs, ks, rank, flags, (cudaStream_t)stream, outs);
  });
}

nuri_status nuri_topk_patterns(nuri_graph* g, int32_t M, int32_t k, int32_t rank,
                               uint32_t flags, void* stream, nuri_result** out) {
  return guarded([&] {
    if (!g || !out) NURI_FAIL(NURI_ERR_INVALID, "nuri_topk_patterns: NULL argument");
    *out = nullptr;
    if (k < 1) NURI_FAIL(NURI_ERR_INVALID, "nuri_topk_patterns: k must be >= 1");
    if (M < 1 || M > 5) NURI_FAIL(NURI_ERR_INVALID, "nuri_topk_patterns: M must be 1..5");
    if (rank != NURI_RANK_MNI) NURI_FAIL(NURI_ERR_INVALID, "nuri_topk_patterns: rank must be NURI_RANK_MNI");
    if (!g->d.labels || !g->d.lsoff) NURI_FAIL(NURI_ERR_INVALID, "nuri_topk_patterns: graph has no labels");
    if (flags & NURI_PATTERNS_EDGE_ORIENTED) topk_patterns_edge(g, M, k, flags, (cudaStream_t)stream, out);
    else topk_patterns(g, M, k, flags, (cudaStream_t)stream, out);
  });
}

}  // extern "C"

namespace nuri {
namespace {

// The first `count` rows of r, or, when count < 0, the rows whose score is at least
// `min_score`; a new result with r's kind and counters.
nuri_result* slice_result(const nuri_result* r, int32_t count, int64_t min_score) {
  if (count < 0) {
    count = 0;
    while (count < r->count && r->score[count] >= min_score) ++count;
  }
  count = std::min(count, r->count);
  const int64_t nv = r->vert_off[count], ne = r->edge_off[count];
  nuri_result* o = new_result(r->kind, count, nv, ne, r->labels != nullptr);
  memcpy(o->score, r->score, sizeof(int64_t) * count);
  memcpy(o->vert_off, r->vert_off, sizeof(int32_t) * (count + 1));
  memcpy(o->edge_off, r->edge_off, sizeof(int32_t) * (count + 1));
  memcpy(o->verts, r->verts, sizeof(int32_t) * nv);
  memcpy(o->edges, r->edges, sizeof(int32_t) * 2 * ne);
  if (r->labels) memcpy(o->labels, r->labels, sizeof(int32_t) * nv);
  o->stats = r->stats;
  return o;
}

// A connected simple query of 1..8 vertices (the isomorphism engine's precondition).
bool query_ok(const nuri_query& q) {
  if (q.nq < 1 || q.nq > 8 || q.ne < 0 || !q.labels || (q.ne > 0 && (!q.src || !q.dst)))
    return false;
  uint32_t adj[8] = {};
  for (int e = 0; e < q.ne; ++e) {
    const int a = q.src[e], b = q.dst[e];
    if (a < 0 || b < 0 || a >= q.nq || b >= q.nq || a == b) return false;
    adj[a] |= 1u << b;
    adj[b] |= 1u << a;
  }
  uint32_t seen = 1, frontier = 1;
  while (frontier) {
    uint32_t nxt = 0;
    for (int v = 0; v < q.nq; ++v)
      if ((frontier >> v) & 1) nxt |= adj[v];
    frontier = nxt & ~seen;
    seen |= nxt;
  }
  return seen == (1u << q.nq) - 1;
}

// Requests of one shared-work group (same kind and key), answered by one run of the
// largest k: cliques and patterns.
template <class Run>
void run_prefix_group(const std::vector<int>& idx, const nuri_request* reqs, uint32_t flags,
                      Run&& run, nuri_result** outs) {
  int32_t K = 0;
  for (int i : idx) K = std::max(K, reqs[i].k);
  nuri_result* r = nullptr;
  run(K, flags, &r);
  struct Free {
    nuri_result* r;
    ~Free() { nuri_free_result(r); }
  } guard{r};
  const bool ties = flags & NURI_KEEP_TIES;
  for (int i : idx) {
    const int32_t k = reqs[i].k;
    if (!ties) outs[i] = slice_result(r, k, 0);
    else if (r->count < k) outs[i] = slice_result(r, r->count, 0);
    else outs[i] = slice_result(r, -1, r->score[k - 1]);  // every row tied with the k-th
  }
}

}  // namespace
}  // namespace nuri

extern "C" {

nuri_status nuri_topk_batch(nuri_graph* g, int32_t nreq, const nuri_request* reqs,
                            void* stream, nuri_result** outs) {
  return guarded([&] {
    if (!g || !reqs || !outs || nreq < 0) NURI_FAIL(NURI_ERR_INVALID, "nuri_topk_batch: NULL argument");
    for (int i = 0; i < nreq; ++i) outs[i] = nullptr;
    for (int i = 0; i < nreq; ++i) {
      const nuri_request& r = reqs[i];
      if (r.k < 1) NURI_FAIL(NURI_ERR_INVALID, "nuri_topk_batch: request %d has k < 1", i);
      if (r.kind == NURI_REQ_CLIQUES) {
        if (r.rank != NURI_RANK_SIZE && r.rank != NURI_RANK_WEIGHT_SUM)
          NURI_FAIL(NURI_ERR_INVALID, "nuri_topk_batch: request %d: clique rank must be SIZE or WEIGHT_SUM", i);
        if (r.rank == NURI_RANK_WEIGHT_SUM && !g->d.weights)
          NURI_FAIL(NURI_ERR_INVALID, "nuri_topk_batch: graph has no weights");
      } else if (r.kind == NURI_REQ_ISO) {
        if (r.rank != NURI_RANK_WEIGHT_SUM && r.rank != NURI_RANK_DEGREE_SUM &&
            r.rank != NURI_RANK_EDGE_WEIGHT_SUM)
          NURI_FAIL(NURI_ERR_INVALID, "nuri_topk_batch: request %d: bad isomorphism rank", i);
        if (!query_ok(r.query)) NURI_FAIL(NURI_ERR_INVALID, "nuri_topk_batch: request %d: bad query", i);
        if (!g->d.labels || !g->d.lsoff) NURI_FAIL(NURI_ERR_INVALID, "nuri_topk_batch: graph has no labels");
        if (r.rank == NURI_RANK_WEIGHT_SUM && !g->d.weights)
          NURI_FAIL(NURI_ERR_INVALID, "nuri_topk_batch: graph has no weights");
        if (r.rank == NURI_RANK_EDGE_WEIGHT_SUM && !g->d.ew)
          NURI_FAIL(NURI_ERR_INVALID, "nuri_topk_batch: graph has no edge weights");
      } else if (r.kind == NURI_REQ_PATTERNS) {
        if (r.rank != NURI_RANK_MNI) NURI_FAIL(NURI_ERR_INVALID, "nuri_topk_batch: request %d: pattern rank must be NURI_RANK_MNI", i);
        if (r.pattern_edges < 1 || r.pattern_edges > 5)
          NURI_FAIL(NURI_ERR_INVALID, "nuri_topk_batch: request %d: M must be 1..5", i);
        if (!g->d.labels || !g->d.lsoff) NURI_FAIL(NURI_ERR_INVALID, "nuri_topk_batch: graph has no labels");
      } else {
        NURI_FAIL(NURI_ERR_INVALID, "nuri_topk_batch: request %d has an unknown kind", i);
      }
    }
    cudaStream_t s = (cudaStream_t)stream;
    // groups: (kind, key) -> request indices, in first-appearance order
    std::vector<std::pair<std::pair<int, uint64_t>, std::vector<int>>> groups;
    for (int i = 0; i < nreq; ++i) {
      const nuri_request& r = reqs[i];
      uint64_t key = r.flags;
      if (r.kind == NURI_REQ_ISO || r.kind == NURI_REQ_CLIQUES)
        key |= (uint64_t)(uint32_t)r.rank << 32;
      if (r.kind == NURI_REQ_PATTERNS) key |= (uint64_t)(uint32_t)r.pattern_edges << 32;
      auto it = std::find_if(groups.begin(), groups.end(), [&](const auto& x) {
        return x.first.first == r.kind && x.first.second == key;
      });
      if (it == groups.end()) groups.push_back({{r.kind, key}, {i}});
      else it->second.push_back(i);
    }
    try {
      for (auto& grp : groups) {
        const std::vector<int>& idx = grp.second;
        const nuri_request& r0 = reqs[idx[0]];
        if (r0.kind == NURI_REQ_CLIQUES) {
          // the ranking is a total order that does not depend on k (by size or by weight,
          // ties by sorted ids): every request is a prefix of the largest one
          const bool weighted = r0.rank == NURI_RANK_WEIGHT_SUM;
          run_prefix_group(idx, reqs, r0.flags, [&](int32_t K, uint32_t fl, nuri_result** o) {
            if (weighted) topk_wcliques(g, K, fl, s, o);
            else topk_cliques(g, K, fl, 0, s, o);
          }, outs);
        } else if (r0.kind == NURI_REQ_PATTERNS) {
          run_prefix_group(idx, reqs, r0.flags, [&](int32_t K, uint32_t fl, nuri_result** o) {
            if (fl & NURI_PATTERNS_EDGE_ORIENTED) topk_patterns_edge(g, r0.pattern_edges, K, fl, s, o);
            else topk_patterns(g, r0.pattern_edges, K, fl, s, o);
          }, outs);
        } else {
          std::vector<nuri_query> qs;
          std::vector<int32_t> ks;
          for (int i : idx) {
            qs.push_back(reqs[i].query);
            ks.push_back(reqs[i].k);
          }
          std::vector<nuri_result*> res(idx.size(), nullptr);
          topk_iso_batch(g, (int32_t)idx.size(), qs.data(), ks.data(), r0.rank, r0.flags, s,
                         res.data());
          for (size_t j = 0; j < idx.size(); ++j) outs[idx[j]] = res[j];
        }
      }
    } catch (...) {
      for (int i = 0; i < nreq; ++i) {
        nuri_free_result(outs[i]);
        outs[i] = nullptr;
      }
      throw;
    }
  });
}

nuri_status nuri_set_partition(nuri_graph* g, const nuri_partition* p) {
  return guarded([&] {
    if (!g) NURI_FAIL(NURI_ERR_INVALID, "nuri_set_partition: NULL graph");
    if (!p || p->count == 1) {
      g->part = nuri_partition{0, 1, nullptr, nullptr};
      return;
    }
    if (p->count < 1 || p->index < 0 || p->index >= p->count)
      NURI_FAIL(NURI_ERR_INVALID, "nuri_set_partition: need 0 <= index < count");
    g->part = *p;
  });
}

int32_t nuri_seed_part(int32_t v, int32_t count) { return seed_part(v, count); }

nuri_status nuri_set_time_budget(double ms) {
  return guarded([&] {
    if (!(ms >= 0.0)) NURI_FAIL(NURI_ERR_INVALID, "nuri_set_time_budget: ms must be >= 0");
    g_budget_ns.store((uint64_t)(ms * 1e6));
  });
}

void nuri_free_result(nuri_result* r) {
  if (!r) return;
  free(r->score);
  free(r->vert_off);
  free(r->verts);
  free(r->edge_off);
  free(r->edges);
  free(r->labels);
  free(r);
}

}  // extern "C"

extern "C" nuri_status nuri_hop_index(nuri_graph* g, int32_t hops, int32_t degree_rank,
                                      int32_t* out, int32_t device_out, void* stream) {
  return guarded([&] {
    if (!g || !out) NURI_FAIL(NURI_ERR_INVALID, "nuri_hop_index: NULL argument");
    if (hops < 1 || hops > g->d.H) NURI_FAIL(NURI_ERR_INVALID, "nuri_hop_index: hops must be in 1..%d", g->d.H);
    const int32_t* src = degree_rank ? g->d.idx_d : g->d.idx_w;
    if (!src) NURI_FAIL(NURI_ERR_INVALID, "nuri_hop_index: index not built");
    cudaStream_t s = (cudaStream_t)stream;
    size_t bytes = sizeof(int32_t) * (size_t)hops * g->d.n * g->d.L;
    NURI_CUDA(cudaMemcpyAsync(out, src, bytes, device_out ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
    NURI_CUDA(cudaStreamSynchronize(s));
  });
}
