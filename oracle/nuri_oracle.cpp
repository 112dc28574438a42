// Nuri oracle -- TEST INFRASTRUCTURE ONLY.
//
// A plain, slow, single-threaded CPU restatement of what the paper's method computes
// (arXiv 1807.08888, "Nuri: An Efficient System for Subgraph Discovery").  It exists to check
// the CUDA library: only the tests, the smoke check and the benchmark's CPU-baseline leg load
// it.  It shares no code, header, table or helper with the CUDA path (it includes nothing from
// the package and the package includes nothing from here).
//
// Contents (each function cites the passage it follows):
//   * graph clean-up: symmetrise, drop self-loops and duplicates (Section 6.1 datasets are
//     undirected; Table 2).
//   * orc_topk_cliques  -- Algorithm 1 (Section 3.2) with the clique user functions of
//     Section 3.2 / Section 4.1 (Listing 1's candidate set P, the Carraghan-Pardalos bound,
//     priority (|V|,|P|)), canonical extension by increasing id (Section 3.2 example).
//   * orc_topk_wcliques -- the same with vertex-weighted ranking (Section 2 top-k semantics:
//     a cumulative weight as the ranking criterion) and the weighted Carraghan-Pardalos bound.
//   * orc_bk_cliques    -- Bron-Kerbosch with pivoting over a degeneracy order: an
//     independent enumeration of maximal cliques used to pin orc_topk_cliques.
//   * orc_hop_index     -- the hop/label max index of Section 4.3 (Listing 3), both by explicit
//     walk-reachability sets (definition) and by the one-hop recurrence.
//   * orc_topk_iso      -- Algorithm 1 with the subgraph-isomorphism user functions of
//     Section 4.3 (score sum, index upper bound u, priority (edges, score+u)).
//   * orc_mni / orc_topk_patterns -- minimum image-based support (Section 2, Bringmann and
//     Nijssen) by existence search per (pattern vertex, data vertex), and Algorithm 2
//     (Section 3.3) over pattern groups with priority (m, f) and dominance f < f(k-th).
//
// Readings of the paper that are not spelled out there (they are listed with reasons in the
// design notes of the repository):
//   * results are ranked by score only (clique size, weight sum, support); the queue priority
//     is the paper's tuple; ties at the k-th place are broken by sorted vertex ids (cliques),
//     sorted vertex ids then sorted edge list (iso), canonical code (patterns);
//   * pruning is strict: prune iff bound < k-th score;
//   * subgraph-isomorphism matches are non-induced images (V_s, E_s); automorphic mappings
//     give the same result once;
//   * index(v, l, h) = max weight over vertices of label l reachable from v by a walk of
//     length 1..h (cumulative hops);
//   * patterns are vertex-labelled, edge-unlabelled, connected, non-induced; the canonical code
//     of a pattern is the minimum over vertex permutations of
//     [n, labels in order, upper-triangle adjacency bits row-major].
//
// Parity unpinned: nothing here reproduces the Fig. 6 bound values (the data graph of that
// figure cannot be recovered from the text).

#include <algorithm>
#include <chrono>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <functional>
#include <map>
#include <queue>
#include <set>
#include <vector>

namespace {

using std::vector;

struct G {
  int n = 0;
  vector<vector<int>> adj;  // sorted, unique, no self loops
  vector<int> lab;          // may be empty
  vector<int64_t> w;        // may be empty
  bool has(int a, int b) const {
    const auto& x = adj[a];
    return std::binary_search(x.begin(), x.end(), b);
  }
};

G build_graph(int n, int64_t m, const int32_t* src, const int32_t* dst) {
  G g;
  g.n = n;
  g.adj.assign(n, {});
  for (int64_t e = 0; e < m; ++e) {
    int a = src[e], b = dst[e];
    if (a == b) continue;
    g.adj[a].push_back(b);
    g.adj[b].push_back(a);
  }
  for (auto& x : g.adj) {
    std::sort(x.begin(), x.end());
    x.erase(std::unique(x.begin(), x.end()), x.end());
  }
  return g;
}

// ---- result marshalling ---------------------------------------------------------------------
struct Row {
  int64_t score = 0;
  vector<int> verts;                      // sorted ascending (cliques, iso) / canonical order
  vector<std::pair<int, int>> edges;      // (min,max) sorted (iso) / canonical pairs (patterns)
  vector<int> labels;                     // patterns: label of each canonical vertex
};

}  // namespace

extern "C" {

typedef struct orc_result {
  int32_t count;
  int64_t* score;
  int32_t* vert_off;
  int32_t* verts;
  int32_t* edge_off;
  int32_t* edges;
  int32_t* labels;
  int64_t expansions;   // children created (one per extension of Algorithm 1 / Algorithm 2)
  int64_t dequeued;     // subgraphs / groups removed from Q
  int64_t pruned;       // children dropped by dominated()
  int32_t complete;     // 0 when a work budget stopped the run early
  double seconds;
} orc_result;

void orc_free(orc_result* r) {
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

namespace {

orc_result* pack(const vector<Row>& rows) {
  orc_result* r = (orc_result*)calloc(1, sizeof(orc_result));
  r->count = (int32_t)rows.size();
  size_t nv = 0, ne = 0;
  for (auto& x : rows) {
    nv += x.verts.size();
    ne += x.edges.size();
  }
  r->score = (int64_t*)malloc(sizeof(int64_t) * (rows.size() + 1));
  r->vert_off = (int32_t*)malloc(sizeof(int32_t) * (rows.size() + 1));
  r->edge_off = (int32_t*)malloc(sizeof(int32_t) * (rows.size() + 1));
  r->verts = (int32_t*)malloc(sizeof(int32_t) * (nv + 1));
  r->labels = (int32_t*)malloc(sizeof(int32_t) * (nv + 1));
  r->edges = (int32_t*)malloc(sizeof(int32_t) * (2 * ne + 2));
  size_t pv = 0, pe = 0;
  for (size_t i = 0; i < rows.size(); ++i) {
    r->score[i] = rows[i].score;
    r->vert_off[i] = (int32_t)pv;
    r->edge_off[i] = (int32_t)pe;
    for (size_t j = 0; j < rows[i].verts.size(); ++j) {
      r->verts[pv] = rows[i].verts[j];
      r->labels[pv] = j < rows[i].labels.size() ? rows[i].labels[j] : -1;
      ++pv;
    }
    for (auto& e : rows[i].edges) {
      r->edges[2 * pe] = e.first;
      r->edges[2 * pe + 1] = e.second;
      ++pe;
    }
  }
  r->vert_off[rows.size()] = (int32_t)pv;
  r->edge_off[rows.size()] = (int32_t)pe;
  r->complete = 1;
  return r;
}

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

// ---- the top-k result set R of Algorithm 1 ----------------------------------------------------
// Entries are kept with their score.  k-th(R) is the k-th largest score among the entries.
// An entry is inserted when |R| < k or its score >= k-th; after an insertion that makes |R| > k,
// every entry with a score below the new k-th score is removed, so ties with the
// k-th entry stay and |R| may exceed k.
template <class Entry>
struct ResultSet {
  int k;
  std::map<int64_t, vector<Entry>, std::greater<int64_t>> by_score;
  int64_t size = 0;
  explicit ResultSet(int k_) : k(k_) {}
  bool full() const { return size >= k; }
  int64_t kth() const {  // only meaningful when full()
    int64_t seen = 0;
    for (auto& kv : by_score) {
      seen += (int64_t)kv.second.size();
      if (seen >= k) return kv.first;
    }
    return INT64_MIN;
  }
  void offer(int64_t score, const Entry& e) {
    if (!(size < k || score >= kth())) return;
    by_score[score].push_back(e);
    ++size;
    if (size > k) {
      int64_t t = kth();
      while (!by_score.empty() && by_score.rbegin()->first < t) {
        size -= (int64_t)by_score.rbegin()->second.size();
        by_score.erase(std::prev(by_score.end()));
      }
    }
  }
};

bool lex_less(const vector<int>& a, const vector<int>& b) {
  return std::lexicographical_compare(a.begin(), a.end(), b.begin(), b.end());
}

// =============================================================================================
// Cliques: Algorithm 1 with the clique user functions (Section 3.2 example, Section 4.1).
//   expandable(s, d) = d in P_s          relevant(s) = true (all cliques) or s is maximal
//   priority(s) = (|V_s|, |P_s|)          dominated(s, o) = |V_s| + |P_s| < |V_o|
// P_s is Listing 1's set (common neighbours of the members) restricted, by the canonical
// extension of Section 3.2 (s2 does not consider v1), to ids above every member.
// =============================================================================================
struct CliqueSub {
  vector<int> V;  // increasing ids
  vector<int> P;  // sorted ids > max(V), adjacent to every member
};

vector<int> common_nbrs_all(const G& g, const vector<int>& V) {
  vector<int> c = g.adj[V[0]];
  for (size_t i = 1; i < V.size(); ++i) {
    vector<int> t;
    std::set_intersection(c.begin(), c.end(), g.adj[V[i]].begin(), g.adj[V[i]].end(),
                          std::back_inserter(t));
    c.swap(t);
  }
  return c;
}

}  // namespace

extern "C" int orc_topk_cliques(int32_t n, int64_t m, const int32_t* src, const int32_t* dst,
                                int32_t k, int32_t maximal_only, int64_t budget,
                                orc_result** out) {
  if (k < 1 || n < 0) return 1;
  double t0 = now_s();
  G g = build_graph(n, m, src, dst);
  struct QE {
    int64_t p0, p1, seq;
    int32_t idx;
  };
  struct Cmp {
    bool operator()(const QE& a, const QE& b) const {
      if (a.p0 != b.p0) return a.p0 < b.p0;
      if (a.p1 != b.p1) return a.p1 < b.p1;
      return a.seq > b.seq;  // FIFO among equal priorities
    }
  };
  vector<CliqueSub> store;
  vector<int32_t> free_slots;
  std::priority_queue<QE, vector<QE>, Cmp> Q;
  int64_t seq = 0;
  auto enqueue = [&](CliqueSub&& s) {
    int32_t slot;
    if (!free_slots.empty()) {
      slot = free_slots.back();
      free_slots.pop_back();
      store[slot] = std::move(s);
    } else {
      slot = (int32_t)store.size();
      store.push_back(std::move(s));
    }
    Q.push({(int64_t)store[slot].V.size(), (int64_t)store[slot].P.size(), seq++, slot});
  };
  // Algorithm 1, initialisation: one unit subgraph per vertex.
  for (int v = 0; v < n; ++v) {
    CliqueSub s;
    s.V = {v};
    for (int u : g.adj[v])
      if (u > v) s.P.push_back(u);
    enqueue(std::move(s));
  }
  ResultSet<vector<int>> R(k);
  int64_t expansions = 0, dequeued = 0, pruned = 0;
  int complete = 1;
  while (!Q.empty()) {                        // until the queue is empty
    QE top = Q.top();                         // dequeue the highest priority
    Q.pop();
    CliqueSub s = std::move(store[top.idx]);
    free_slots.push_back(top.idx);
    ++dequeued;
    int64_t score = (int64_t)s.V.size();
    bool relevant = true;
    if (maximal_only) relevant = common_nbrs_all(g, s.V).empty();
    if (relevant) R.offer(score, s.V);        // result-set update
    // expand unless dominated by the k-th entry
    if (!R.full() || !((int64_t)(s.V.size() + s.P.size()) < R.kth())) {
      for (size_t j = 0; j < s.P.size(); ++j) {  // neighbouring vertices d
        int d = s.P[j];                           // expandable(s, d) = d in P_s
        CliqueSub c;                              // the child s + d
        c.V = s.V;
        c.V.push_back(d);
        for (size_t t = j + 1; t < s.P.size(); ++t)
          if (g.has(d, s.P[t])) c.P.push_back(s.P[t]);
        ++expansions;
        // dominated(s', k-th(R))
        if (!R.full() || !((int64_t)(c.V.size() + c.P.size()) < R.kth()))
          enqueue(std::move(c));                  // enqueue the child
        else
          ++pruned;
      }
    }
    if (budget > 0 && expansions >= budget) {
      complete = 0;
      break;
    }
  }
  vector<Row> rows;
  for (auto& kv : R.by_score)
    for (auto& V : kv.second) {
      Row r;
      r.score = kv.first;
      r.verts = V;
      rows.push_back(r);
    }
  std::sort(rows.begin(), rows.end(), [](const Row& a, const Row& b) {
    if (a.score != b.score) return a.score > b.score;
    return lex_less(a.verts, b.verts);
  });
  if ((int)rows.size() > k) rows.resize(k);
  orc_result* r = pack(rows);
  r->expansions = expansions;
  r->dequeued = dequeued;
  r->pruned = pruned;
  r->complete = complete;
  r->seconds = now_s() - t0;
  *out = r;
  return 0;
}

// =============================================================================================
// Vertex-weighted cliques: Algorithm 1 with the clique user functions above, ranked by the
// other criterion Section 2's top-k semantics allows, a cumulative weight: score(s) = sum of
// w(v) over V_s (weights >= 0).  The bound follows the Carraghan-Pardalos one with weights:
// every clique below s adds a subset of P_s, so dominated(s, o) = w(V_s) + w(P_s) < score(o).
//   priority(s) = (w(V_s) + w(P_s), w(V_s))      (best bound first; it orders work only)
// Ties at the k-th place are broken by sorted ids, as for sizes.
// =============================================================================================
extern "C" int orc_topk_wcliques(int32_t n, int64_t m, const int32_t* src, const int32_t* dst,
                                 const int32_t* weights, int32_t k, int32_t maximal_only,
                                 int64_t budget, orc_result** out) {
  if (k < 1 || n < 0 || (n > 0 && !weights)) return 1;
  for (int v = 0; v < n; ++v)
    if (weights[v] < 0) return 1;
  double t0 = now_s();
  G g = build_graph(n, m, src, dst);
  auto wsum = [&](const vector<int>& S) {
    int64_t t = 0;
    for (int v : S) t += weights[v];
    return t;
  };
  struct QE {
    int64_t p0, p1, seq;
    int32_t idx;
  };
  struct Cmp {
    bool operator()(const QE& a, const QE& b) const {
      if (a.p0 != b.p0) return a.p0 < b.p0;
      if (a.p1 != b.p1) return a.p1 < b.p1;
      return a.seq > b.seq;
    }
  };
  struct WSub {
    CliqueSub s;
    int64_t wv, wp;  // w(V_s), w(P_s)
  };
  vector<WSub> store;
  vector<int32_t> free_slots;
  std::priority_queue<QE, vector<QE>, Cmp> Q;
  int64_t seq = 0;
  auto enqueue = [&](WSub&& x) {
    int32_t slot;
    if (!free_slots.empty()) {
      slot = free_slots.back();
      free_slots.pop_back();
      store[slot] = std::move(x);
    } else {
      slot = (int32_t)store.size();
      store.push_back(std::move(x));
    }
    Q.push({store[slot].wv + store[slot].wp, store[slot].wv, seq++, slot});
  };
  for (int v = 0; v < n; ++v) {
    WSub x;
    x.s.V = {v};
    for (int u : g.adj[v])
      if (u > v) x.s.P.push_back(u);
    x.wv = weights[v];
    x.wp = wsum(x.s.P);
    enqueue(std::move(x));
  }
  ResultSet<vector<int>> R(k);
  int64_t expansions = 0, dequeued = 0, pruned = 0;
  int complete = 1;
  while (!Q.empty()) {
    QE top = Q.top();
    Q.pop();
    WSub x = std::move(store[top.idx]);
    free_slots.push_back(top.idx);
    ++dequeued;
    bool relevant = true;
    if (maximal_only) relevant = common_nbrs_all(g, x.s.V).empty();
    if (relevant) R.offer(x.wv, x.s.V);
    if (!R.full() || !(x.wv + x.wp < R.kth())) {
      for (size_t j = 0; j < x.s.P.size(); ++j) {
        int d = x.s.P[j];
        WSub c;
        c.s.V = x.s.V;
        c.s.V.push_back(d);
        for (size_t t = j + 1; t < x.s.P.size(); ++t)
          if (g.has(d, x.s.P[t])) c.s.P.push_back(x.s.P[t]);
        c.wv = x.wv + weights[d];
        c.wp = wsum(c.s.P);
        ++expansions;
        if (!R.full() || !(c.wv + c.wp < R.kth())) enqueue(std::move(c));
        else ++pruned;
      }
    }
    if (budget > 0 && expansions >= budget) {
      complete = 0;
      break;
    }
  }
  vector<Row> rows;
  for (auto& kv : R.by_score)
    for (auto& V : kv.second) {
      Row r;
      r.score = kv.first;
      r.verts = V;
      rows.push_back(r);
    }
  std::sort(rows.begin(), rows.end(), [](const Row& a, const Row& b) {
    if (a.score != b.score) return a.score > b.score;
    return lex_less(a.verts, b.verts);
  });
  if ((int)rows.size() > k) rows.resize(k);
  orc_result* r = pack(rows);
  r->expansions = expansions;
  r->dequeued = dequeued;
  r->pruned = pruned;
  r->complete = complete;
  r->seconds = now_s() - t0;
  *out = r;
  return 0;
}

// =============================================================================================
// Bron-Kerbosch with pivoting over a degeneracy order: every maximal clique exactly once.  mode 1: top-k maximal cliques by (size desc, ids lex asc).  mode 0: top-k of all
// cliques, obtained as the distinct subsets of maximal cliques, size by size from the largest
// (refuses inputs where a size level would need more than 2e7 subsets).
// =============================================================================================
namespace {

struct BK {
  const G& g;
  std::function<void(const vector<int>&)> report;
  explicit BK(const G& gg) : g(gg) {}
  vector<int> inter(const vector<int>& a, const vector<int>& b) {
    vector<int> t;
    std::set_intersection(a.begin(), a.end(), b.begin(), b.end(), std::back_inserter(t));
    return t;
  }
  void rec(vector<int>& Rv, vector<int> P, vector<int> X) {
    if (P.empty() && X.empty()) {
      vector<int> c = Rv;
      std::sort(c.begin(), c.end());
      report(c);
      return;
    }
    if (P.empty()) return;  // X non-empty: R is not maximal
    // pivot: the vertex of P with most neighbours in P (any pivot keeps the enumeration
    // exact; taking it from P keeps the cost proportional to |P|^2 when X is large)
    int best = -1;
    size_t bestc = 0;
    for (int u : P) {
      size_t c = 0;
      for (int p : P) c += g.has(u, p) ? 1 : 0;
      if (best < 0 || c > bestc) {
        best = u;
        bestc = c;
      }
    }
    vector<int> cand;
    std::set_difference(P.begin(), P.end(), g.adj[best].begin(), g.adj[best].end(),
                        std::back_inserter(cand));
    for (int v : cand) {
      Rv.push_back(v);
      rec(Rv, inter(P, g.adj[v]), inter(X, g.adj[v]));
      Rv.pop_back();
      P.erase(std::lower_bound(P.begin(), P.end(), v));
      X.insert(std::lower_bound(X.begin(), X.end(), v), v);
    }
  }
  void run() {
    // degeneracy order by repeatedly removing a minimum-degree vertex
    int n = g.n;
    vector<int> deg(n);
    std::set<std::pair<int, int>> heap;
    for (int v = 0; v < n; ++v) {
      deg[v] = (int)g.adj[v].size();
      heap.insert({deg[v], v});
    }
    vector<int> pos(n, -1), order;
    order.reserve(n);
    while (!heap.empty()) {
      auto it = heap.begin();
      int v = it->second;
      heap.erase(it);
      pos[v] = (int)order.size();
      order.push_back(v);
      for (int u : g.adj[v])
        if (pos[u] < 0) {
          heap.erase({deg[u], u});
          --deg[u];
          heap.insert({deg[u], u});
        }
    }
    for (int v : order) {
      vector<int> P, X;
      for (int u : g.adj[v]) (pos[u] > pos[v] ? P : X).push_back(u);
      vector<int> Rv = {v};
      rec(Rv, P, X);
    }
  }
};

struct RowKeyLess {
  bool operator()(const vector<int>& a, const vector<int>& b) const {
    if (a.size() != b.size()) return a.size() > b.size();
    return lex_less(a, b);
  }
};

}  // namespace

extern "C" int orc_bk_cliques(int32_t n, int64_t m, const int32_t* src, const int32_t* dst,
                              int32_t k, int32_t mode, orc_result** out) {
  if (k < 1 || n < 0) return 1;
  double t0 = now_s();
  G g = build_graph(n, m, src, dst);
  BK bk(g);
  vector<Row> rows;
  if (mode == 1) {
    std::set<vector<int>, RowKeyLess> top;
    bk.report = [&](const vector<int>& c) {
      top.insert(c);
      if ((int)top.size() > k) top.erase(std::prev(top.end()));
    };
    bk.run();
    for (auto& c : top) {
      Row r;
      r.score = (int64_t)c.size();
      r.verts = c;
      rows.push_back(r);
    }
  } else {
    vector<vector<int>> maxi;
    bk.report = [&](const vector<int>& c) { maxi.push_back(c); };
    bk.run();
    size_t omega = 0;
    for (auto& c : maxi) omega = std::max(omega, c.size());
    for (size_t s = omega; s >= 1 && (int)rows.size() < k; --s) {
      std::set<vector<int>> level;
      for (auto& c : maxi) {
        if (c.size() < s) continue;
        // all s-subsets of c, in lexicographic order of index tuples
        vector<int> idx(s);
        for (size_t i = 0; i < s; ++i) idx[i] = (int)i;
        while (true) {
          vector<int> sub(s);
          for (size_t i = 0; i < s; ++i) sub[i] = c[idx[i]];
          level.insert(sub);
          if (level.size() > 20000000) return 2;
          int i = (int)s - 1;
          while (i >= 0 && idx[i] == (int)(c.size() - s + i)) --i;
          if (i < 0) break;
          ++idx[i];
          for (size_t j = i + 1; j < s; ++j) idx[j] = idx[j - 1] + 1;
        }
      }
      for (auto& sub : level) {
        if ((int)rows.size() >= k) break;
        Row r;
        r.score = (int64_t)s;
        r.verts = sub;
        rows.push_back(r);
      }
      if (s == 1) break;
    }
  }
  orc_result* r = pack(rows);
  r->seconds = now_s() - t0;
  *out = r;
  return 0;
}

// =============================================================================================
// Hop/label max index (Section 4.3, Listing 3), cumulative reading:
//   index(v, l, h) = max w(x) over x with label l reachable from v by a walk of length 1..h,
//   or -1 when there is none (weights are non-negative).
// method 0 computes it from the definition with explicit reachability sets (small graphs);
// method 1 uses the one-hop recurrence index_h(v) = max over x in N(v) of
//   max(own(x), index_{h-1}(x)), own(x) = w(x) in slot label(x).
// Output layout: out[((h-1) * n + v) * L + l], h = 1..H.
// =============================================================================================
extern "C" int orc_hop_index(int32_t n, int64_t m, const int32_t* src, const int32_t* dst,
                             const uint8_t* labels, const int32_t* weights, int32_t L,
                             int32_t H, int32_t method, int32_t* out) {
  if (H < 1 || L < 1 || !labels || !weights) return 1;
  G g = build_graph(n, m, src, dst);
  if (method == 0) {
    for (int v = 0; v < n; ++v) {
      vector<char> cur(n, 0), seen(n, 0);
      cur[v] = 1;
      for (int h = 1; h <= H; ++h) {
        vector<char> nxt(n, 0);
        for (int x = 0; x < n; ++x)
          if (cur[x])
            for (int y : g.adj[x]) nxt[y] = 1;
        for (int x = 0; x < n; ++x)
          if (nxt[x]) seen[x] = 1;
        cur.swap(nxt);
        for (int l = 0; l < L; ++l) {
          int32_t best = -1;
          for (int x = 0; x < n; ++x)
            if (seen[x] && labels[x] == l) best = std::max(best, weights[x]);
          out[((int64_t)(h - 1) * n + v) * L + l] = best;
        }
      }
    }
    return 0;
  }
  vector<int32_t> prev((int64_t)n * L, -1), cur((int64_t)n * L, -1);
  for (int h = 1; h <= H; ++h) {
    for (int v = 0; v < n; ++v)
      for (int l = 0; l < L; ++l) {
        int32_t best = -1;
        for (int x : g.adj[v]) {
          if (labels[x] == l) best = std::max(best, weights[x]);
          best = std::max(best, prev[(int64_t)x * L + l]);
        }
        cur[(int64_t)v * L + l] = best;
      }
    std::memcpy(out + (int64_t)(h - 1) * n * L, cur.data(), sizeof(int32_t) * n * L);
    prev.swap(cur);
  }
  return 0;
}

// =============================================================================================
// Subgraph isomorphism: Algorithm 1 with the user functions of Section 4.3.
//   A subgraph is a partial mapping of the query, grown one query vertex at a time along a
//   breadth-first order of the query from its root (each step adds the vertex with the query
//   edges to already-matched vertices; expandable() admits only images that keep the partial
//   subgraph isomorphic to the matched part of the query -- Ullmann-style targeted expansion).
//   score = sum of vertex scores (weights, or degrees when rank == 1);
//   u = sum over unmatched q of index(mu(root), label(q), hop(q));
//   rank == 2 ranks by the other criterion that Section 2's top-k semantics names, the
//   cumulative edge weight: score = sum of w(e) over the image's edges E_s (the data edges the
//   query edges land on), u = (query edges not yet matched) x (largest edge weight), a valid
//   bound since every unmatched query edge adds one data edge of weight at most that.
//   Edge weights ew[e] belong to the input pair (src[e], dst[e]); an undirected edge given by
//   several pairs takes the largest of their weights; pairs without a weight of their own do
//   not exist (every pair carries one).
//   priority = (matched query edges, score + u);  dominated(s, o) = score + u < score(o);
//   relevant(s) = every query vertex is matched.  Automorphic mappings with the same image are
//   one subgraph: an image already in R is not inserted again.
// rank: 0 = weight sum, 1 = degree sum, 2 = edge-weight sum.  H_avail: number of index hops to use (>= query radius
// is exact; hops beyond it use the per-label global maximum, which is also a valid bound).
// induced != 0: the other reading of Section 2's definition (an edge between two images iff
// there is one between the query vertices): expandable() also rejects an image adjacent to the
// image of an already-matched query vertex that is not adjacent to the new one.
// =============================================================================================
extern "C" int orc_topk_iso(int32_t n, int64_t m, const int32_t* src, const int32_t* dst,
                            const uint8_t* labels, const int32_t* weights,
                            const int32_t* edge_w, int32_t rank,
                            int32_t nq, const uint8_t* qlab, int32_t qne, const int32_t* qsrc,
                            const int32_t* qdst, int32_t k, int64_t budget, int32_t induced,
                            orc_result** out) {
  if (k < 1 || nq < 1 || nq > 8 || !labels) return 1;
  if (rank == 0 && !weights) return 1;
  if (rank == 2 && !edge_w) return 1;
  if (rank < 0 || rank > 2) return 1;
  double t0 = now_s();
  G g = build_graph(n, m, src, dst);
  vector<int64_t> score_of(n, 0);
  if (rank != 2)
    for (int v = 0; v < n; ++v) score_of[v] = rank == 1 ? (int64_t)g.adj[v].size() : weights[v];
  // edge weights (rank 2): the largest weight given for each undirected edge
  std::map<std::pair<int, int>, int64_t> wedge;
  int64_t wmax = 0;
  if (rank == 2)
    for (int64_t e = 0; e < m; ++e) {
      const int a = src[e], b = dst[e];
      if (a == b) continue;
      if (edge_w[e] < 0) return 1;
      auto key = std::make_pair(std::min(a, b), std::max(a, b));
      auto it = wedge.find(key);
      if (it == wedge.end()) wedge[key] = edge_w[e];
      else it->second = std::max(it->second, (int64_t)edge_w[e]);
      wmax = std::max(wmax, (int64_t)edge_w[e]);
    }
  auto wof = [&](int a, int b) -> int64_t {
    return wedge.at(std::make_pair(std::min(a, b), std::max(a, b)));
  };
  int qedges = 0;
  // query adjacency
  vector<vector<int>> qadj(nq, vector<int>(nq, 0));
  for (int e = 0; e < qne; ++e) {
    int a = qsrc[e], b = qdst[e];
    if (a < 0 || b < 0 || a >= nq || b >= nq || a == b) return 1;
    qadj[a][b] = qadj[b][a] = 1;
  }
  for (int a = 0; a < nq; ++a)
    for (int b = a + 1; b < nq; ++b) qedges += qadj[a][b];
  auto bfs = [&](int r, vector<int>& dist, vector<int>& order, vector<int>& par) {
    dist.assign(nq, -1);
    par.assign(nq, -1);
    order.clear();
    dist[r] = 0;
    order.push_back(r);
    for (size_t i = 0; i < order.size(); ++i) {
      int a = order[i];
      for (int b = 0; b < nq; ++b)
        if (qadj[a][b] && dist[b] < 0) {
          dist[b] = dist[a] + 1;
          par[b] = a;
          order.push_back(b);
        }
    }
  };
  // root = minimum eccentricity, lowest index on ties
  int root = -1, best_ecc = 1 << 30;
  vector<int> dist, order, par;
  for (int r = 0; r < nq; ++r) {
    bfs(r, dist, order, par);
    if ((int)order.size() != nq) return 1;  // disconnected query
    int ecc = *std::max_element(dist.begin(), dist.end());
    if (ecc < best_ecc) {
      best_ecc = ecc;
      root = r;
    }
  }
  bfs(root, dist, order, par);
  int H = best_ecc;
  int L = 0;
  for (int v = 0; v < n; ++v) L = std::max(L, (int)labels[v] + 1);
  for (int q = 0; q < nq; ++q) L = std::max(L, (int)qlab[q] + 1);
  // index by the one-hop recurrence (pinned against the walk-set definition in the tests)
  vector<vector<int64_t>> idx(H + 1, vector<int64_t>((int64_t)n * L, -1));
  for (int h = 1; h <= H; ++h)
    for (int v = 0; v < n; ++v)
      for (int x : g.adj[v])
        for (int l = 0; l < L; ++l) {
          int64_t own = (labels[x] == l) ? score_of[x] : -1;
          int64_t val = std::max(own, idx[h - 1][(int64_t)x * L + l]);
          int64_t& d = idx[h][(int64_t)v * L + l];
          d = std::max(d, val);
        }
  const int64_t NONE = -(int64_t)1 << 40;
  struct IsoSub {
    int depth;  // number of matched query vertices, in BFS order
    int map[8];
    int64_t score, bound;
  };
  auto edges_matched = [&](int depth) {
    int c = 0;
    for (int i = 0; i < depth; ++i)
      for (int j = i + 1; j < depth; ++j) c += qadj[order[i]][order[j]];
    return c;
  };
  auto upper = [&](const IsoSub& s) -> int64_t {
    if (rank == 2) return s.score + (int64_t)(qedges - edges_matched(s.depth)) * wmax;
    int64_t u = 0;
    for (int i = s.depth; i < nq; ++i) {
      int q = order[i];
      int64_t v = idx[dist[q]][(int64_t)s.map[0] * L + qlab[q]];
      if (v < 0) return NONE;
      u += v;
    }
    return s.score + u;
  };
  struct QE {
    int64_t p0, p1, seq;
    int32_t idx;
  };
  struct Cmp {
    bool operator()(const QE& a, const QE& b) const {
      if (a.p0 != b.p0) return a.p0 < b.p0;
      if (a.p1 != b.p1) return a.p1 < b.p1;
      return a.seq > b.seq;
    }
  };
  vector<IsoSub> store;
  vector<int32_t> free_slots;
  std::priority_queue<QE, vector<QE>, Cmp> Q;
  int64_t seq = 0;
  auto enqueue = [&](const IsoSub& s) {
    int32_t slot;
    if (!free_slots.empty()) {
      slot = free_slots.back();
      free_slots.pop_back();
      store[slot] = s;
    } else {
      slot = (int32_t)store.size();
      store.push_back(s);
    }
    Q.push({edges_matched(s.depth), s.bound, seq++, slot});
  };
  for (int v = 0; v < n; ++v) {
    if (labels[v] != qlab[root]) continue;
    IsoSub s{};
    s.depth = 1;
    s.map[0] = v;
    s.score = score_of[v];
    s.bound = upper(s);
    enqueue(s);
  }
  typedef std::pair<vector<int>, vector<std::pair<int, int>>> Image;
  ResultSet<Image> R(k);
  std::set<Image> seen;
  int64_t expansions = 0, dequeued = 0, pruned = 0;
  int complete = 1;
  while (!Q.empty()) {
    QE top = Q.top();
    Q.pop();
    IsoSub s = store[top.idx];
    free_slots.push_back(top.idx);
    ++dequeued;
    if (s.depth == nq) {  // relevant
      Image im;
      for (int i = 0; i < nq; ++i) im.first.push_back(s.map[i]);
      std::sort(im.first.begin(), im.first.end());
      for (int i = 0; i < nq; ++i)
        for (int j = i + 1; j < nq; ++j)
          if (qadj[order[i]][order[j]]) {
            int a = s.map[i], b = s.map[j];
            im.second.push_back({std::min(a, b), std::max(a, b)});
          }
      std::sort(im.second.begin(), im.second.end());
      if (!seen.count(im)) {
        seen.insert(im);
        R.offer(s.score, im);
      }
      continue;
    }
    if (R.full() && s.bound < R.kth()) continue;  // dominated: no expansion
    int q = order[s.depth];
    int pidx = -1;
    for (int i = 0; i < s.depth; ++i)
      if (order[i] == par[q]) pidx = i;
    int anchor = s.map[pidx];
    for (int x : g.adj[anchor]) {
      if (labels[x] != qlab[q]) continue;
      bool ok = true;
      for (int i = 0; i < s.depth && ok; ++i) {
        if (s.map[i] == x) ok = false;
        else if (qadj[q][order[i]] && !g.has(x, s.map[i])) ok = false;
        else if (induced && !qadj[q][order[i]] && g.has(x, s.map[i])) ok = false;
      }
      if (!ok) continue;
      IsoSub c = s;
      c.map[c.depth] = x;
      c.depth += 1;
      c.score = s.score + score_of[x];
      if (rank == 2)  // the query edges from q to the matched vertices land on these edges
        for (int i = 0; i < s.depth; ++i)
          if (qadj[q][order[i]]) c.score += wof(x, s.map[i]);
      c.bound = upper(c);
      ++expansions;
      if (!R.full() || !(c.bound < R.kth())) enqueue(c);
      else ++pruned;
    }
    if (budget > 0 && expansions >= budget) {
      complete = 0;
      break;
    }
  }
  vector<Row> rows;
  for (auto& kv : R.by_score)
    for (auto& im : kv.second) {
      Row r;
      r.score = kv.first;
      r.verts = im.first;
      r.edges = im.second;
      rows.push_back(r);
    }
  std::sort(rows.begin(), rows.end(), [](const Row& a, const Row& b) {
    if (a.score != b.score) return a.score > b.score;
    if (a.verts != b.verts) return lex_less(a.verts, b.verts);
    return a.edges < b.edges;
  });
  if ((int)rows.size() > k) rows.resize(k);
  orc_result* r = pack(rows);
  r->expansions = expansions;
  r->dequeued = dequeued;
  r->pruned = pruned;
  r->complete = complete;
  r->seconds = now_s() - t0;
  *out = r;
  return 0;
}

// =============================================================================================
// Patterns: connected, vertex-labelled, edge-unlabelled graphs with <= 6 vertices.
// =============================================================================================
namespace {

struct Pat {
  int nv = 0;
  vector<int> lab;
  vector<std::pair<int, int>> E;  // a < b
  bool adj(int a, int b) const {
    if (a > b) std::swap(a, b);
    return std::find(E.begin(), E.end(), std::make_pair(a, b)) != E.end();
  }
};

// canonical code: min over vertex permutations of [nv, labels..., upper-triangle bits...]
vector<int> code_of(const Pat& p, vector<int>* best_perm = nullptr) {
  vector<int> perm(p.nv);
  for (int i = 0; i < p.nv; ++i) perm[i] = i;
  vector<vector<int>> A(p.nv, vector<int>(p.nv, 0));
  for (auto& e : p.E) A[e.first][e.second] = A[e.second][e.first] = 1;
  vector<int> best;
  do {
    vector<int> c;
    c.push_back(p.nv);
    for (int j = 0; j < p.nv; ++j) c.push_back(p.lab[perm[j]]);
    for (int a = 0; a < p.nv; ++a)
      for (int b = a + 1; b < p.nv; ++b) c.push_back(A[perm[a]][perm[b]]);
    if (best.empty() || c < best) {
      best = c;
      if (best_perm) *best_perm = perm;
    }
  } while (std::next_permutation(perm.begin(), perm.end()));
  return best;
}

Pat canonical(const Pat& p) {
  vector<int> perm;
  code_of(p, &perm);
  vector<int> inv(p.nv);
  for (int j = 0; j < p.nv; ++j) inv[perm[j]] = j;
  Pat q;
  q.nv = p.nv;
  q.lab.resize(p.nv);
  for (int j = 0; j < p.nv; ++j) q.lab[j] = p.lab[perm[j]];
  for (auto& e : p.E) {
    int a = inv[e.first], b = inv[e.second];
    q.E.push_back({std::min(a, b), std::max(a, b)});
  }
  std::sort(q.E.begin(), q.E.end());
  return q;
}

// Is there an injective, label- and edge-preserving map of p into g with i -> u ?
struct Exist {
  const G& g;
  const Pat& p;
  vector<int> order, parent;
  vector<int> mp;
  vector<char> used_mark;
  Exist(const G& gg, const Pat& pp, int i) : g(gg), p(pp) {
    vector<int> seen(p.nv, 0);
    parent.assign(p.nv, -1);
    order.push_back(i);
    seen[i] = 1;
    for (size_t t = 0; t < order.size(); ++t)
      for (int b = 0; b < p.nv; ++b)
        if (!seen[b] && p.adj(order[t], b)) {
          seen[b] = 1;
          parent[b] = order[t];
          order.push_back(b);
        }
    mp.assign(p.nv, -1);
  }
  bool rec(size_t d) {
    if (d == order.size()) return true;
    int q = order[d];
    int anchor = mp[parent[q]];
    for (int x : g.adj[anchor]) {
      if (g.lab[x] != p.lab[q]) continue;
      bool ok = true;
      for (size_t t = 0; t < d && ok; ++t) {
        int a = order[t];
        if (mp[a] == x) ok = false;
        else if (p.adj(q, a) && !g.has(x, mp[a])) ok = false;
      }
      if (!ok) continue;
      mp[q] = x;
      if (rec(d + 1)) return true;
      mp[q] = -1;
    }
    return false;
  }
  bool from(int u) {
    if (g.lab[u] != p.lab[order[0]]) return false;
    std::fill(mp.begin(), mp.end(), -1);
    mp[order[0]] = u;
    return rec(1);
  }
};

// minimum image-based support (Section 2): min over pattern vertices of the number of
// distinct data vertices that some embedding maps it to.
int64_t mni(const G& g, const Pat& p, vector<int64_t>* dom = nullptr) {
  int64_t f = INT64_MAX;
  if (dom) dom->assign(p.nv, 0);
  for (int i = 0; i < p.nv; ++i) {
    Exist ex(g, p, i);
    int64_t c = 0;
    for (int u = 0; u < g.n; ++u)
      if (ex.from(u)) ++c;
    if (dom) (*dom)[i] = c;
    f = std::min(f, c);
  }
  return f;
}

}  // namespace

extern "C" int orc_mni(int32_t n, int64_t m, const int32_t* src, const int32_t* dst,
                       const uint8_t* labels, int32_t pnv, const int32_t* plab, int32_t pne,
                       const int32_t* psrc, const int32_t* pdst, int64_t* f_out,
                       int64_t* dom_out) {
  if (!labels || pnv < 1 || pnv > 8) return 1;
  G g = build_graph(n, m, src, dst);
  g.lab.assign(labels, labels + n);
  Pat p;
  p.nv = pnv;
  p.lab.assign(plab, plab + pnv);
  for (int e = 0; e < pne; ++e) {
    int a = psrc[e], b = pdst[e];
    if (a == b || a < 0 || b < 0 || a >= pnv || b >= pnv) return 1;
    p.E.push_back({std::min(a, b), std::max(a, b)});
  }
  std::sort(p.E.begin(), p.E.end());
  p.E.erase(std::unique(p.E.begin(), p.E.end()), p.E.end());
  vector<int64_t> dom;
  *f_out = mni(g, p, &dom);
  if (dom_out)
    for (int i = 0; i < pnv; ++i) dom_out[i] = dom[i];
  return 0;
}

// Algorithm 2 over pattern groups (Section 3.3, Section 4.2 user functions):
//   key(s) = pattern(s) (canonical form), relevant(S) = m(S) == M, priority(S) = (m(S), f(S)),
//   dominated(S, O) = f(S) < f(O), expandable(s, d) = edgeCount(s) < M.
// A group is represented by its pattern; its frequency f is the MNI of the pattern, which is
// what Listing 2 aggregates over the group's member subgraphs.  The child groups of S are the
// patterns obtained by adding one data edge next to a member subgraph: a new vertex of any
// label attached to a pattern vertex, or an edge between two pattern vertices; a child group
// exists when the child pattern has at least one embedding.  Every pattern is constructed once
// (the role of gSpan's minimal-DFS-code rule, Property 1).
extern "C" int orc_topk_patterns(int32_t n, int64_t m, const int32_t* src, const int32_t* dst,
                                 const uint8_t* labels, int32_t M, int32_t k,
                                 orc_result** out) {
  if (!labels || M < 1 || M > 5 || k < 1) return 1;
  double t0 = now_s();
  G g = build_graph(n, m, src, dst);
  g.lab.assign(labels, labels + n);
  int L = 0;
  for (int v = 0; v < n; ++v) L = std::max(L, (int)labels[v] + 1);
  struct GroupE {
    Pat p;
    int64_t f;
  };
  struct QE {
    int64_t p0, p1, seq;
    int32_t idx;
  };
  struct Cmp {
    bool operator()(const QE& a, const QE& b) const {
      if (a.p0 != b.p0) return a.p0 < b.p0;
      if (a.p1 != b.p1) return a.p1 < b.p1;
      return a.seq > b.seq;
    }
  };
  vector<GroupE> store;
  std::priority_queue<QE, vector<QE>, Cmp> Q;
  std::set<vector<int>> constructed;
  int64_t seq = 0, expansions = 0, dequeued = 0, pruned = 0;
  ResultSet<vector<int>> R(k);  // entries: canonical codes
  std::map<vector<int>, Pat> pat_of;
  // Algorithm 2, initialisation: one group per 1-edge pattern present in the graph
  {
    std::set<std::pair<int, int>> lp;
    for (int v = 0; v < n; ++v)
      for (int u : g.adj[v]) lp.insert({std::min(labels[v], labels[u]), std::max(labels[v], labels[u])});
    for (auto& x : lp) {
      Pat p;
      p.nv = 2;
      p.lab = {x.first, x.second};
      p.E = {{0, 1}};
      Pat c = canonical(p);
      vector<int> code = code_of(c);
      if (constructed.count(code)) continue;
      constructed.insert(code);
      int64_t f = mni(g, c);
      store.push_back({c, f});
      Q.push({1, f, seq++, (int32_t)store.size() - 1});
    }
  }
  while (!Q.empty()) {
    QE top = Q.top();
    Q.pop();
    const GroupE S = store[top.idx];
    ++dequeued;
    int mS = (int)S.p.E.size();
    vector<int> code = code_of(S.p);
    if (mS == M) {
      pat_of[code] = S.p;
      R.offer(S.f, code);
    }
    if (R.full() && S.f < R.kth()) continue;  // dominated: no expansion
    if (mS >= M) continue;                     // expandable() is false for every member
    // child groups: patterns with one more edge
    vector<Pat> kids;
    for (int i = 0; i < S.p.nv; ++i) {
      if (S.p.nv < 8)
        for (int l = 0; l < L; ++l) {  // forward edge to a new vertex labelled l
          Pat c = S.p;
          c.lab.push_back(l);
          c.E.push_back({i, c.nv});
          c.nv += 1;
          kids.push_back(c);
        }
      for (int j = i + 1; j < S.p.nv; ++j)  // backward edge between pattern vertices
        if (!S.p.adj(i, j)) {
          Pat c = S.p;
          c.E.push_back({i, j});
          std::sort(c.E.begin(), c.E.end());
          kids.push_back(c);
        }
    }
    for (auto& c0 : kids) {
      Pat c = canonical(c0);
      vector<int> cc = code_of(c);
      if (constructed.count(cc)) continue;
      constructed.insert(cc);
      int64_t f = mni(g, c);
      if (f == 0) continue;  // no member subgraph: no group
      ++expansions;
      // enqueue the child group
      if (!R.full() || !(f < R.kth())) {
        store.push_back({c, f});
        Q.push({(int64_t)c.E.size(), f, seq++, (int32_t)store.size() - 1});
      } else {
        ++pruned;
      }
    }
  }
  vector<Row> rows;
  for (auto& kv : R.by_score)
    for (auto& code : kv.second) {
      const Pat& p = pat_of[code];
      Row r;
      r.score = kv.first;
      for (int j = 0; j < p.nv; ++j) r.verts.push_back(j);
      r.labels = p.lab;
      r.edges = p.E;
      rows.push_back(r);
    }
  // tie-break on the canonical code
  std::sort(rows.begin(), rows.end(), [&](const Row& a, const Row& b) {
    if (a.score != b.score) return a.score > b.score;
    Pat pa, pb;
    pa.nv = (int)a.verts.size();
    pa.lab = a.labels;
    pa.E = a.edges;
    pb.nv = (int)b.verts.size();
    pb.lab = b.labels;
    pb.E = b.edges;
    return code_of(pa) < code_of(pb);
  });
  if ((int)rows.size() > k) rows.resize(k);
  orc_result* r = pack(rows);
  r->expansions = expansions;
  r->dequeued = dequeued;
  r->pruned = pruned;
  r->seconds = now_s() - t0;
  *out = r;
  return 0;
}

extern "C" int orc_canonical_code(int32_t pnv, const int32_t* plab, int32_t pne,
                                  const int32_t* psrc, const int32_t* pdst, int32_t* code_out,
                                  int32_t* perm_out) {
  if (pnv < 1 || pnv > 8) return 1;
  Pat p;
  p.nv = pnv;
  p.lab.assign(plab, plab + pnv);
  for (int e = 0; e < pne; ++e) p.E.push_back({std::min(psrc[e], pdst[e]), std::max(psrc[e], pdst[e])});
  vector<int> perm;
  vector<int> c = code_of(p, &perm);
  for (size_t i = 0; i < c.size(); ++i) code_out[i] = c[i];
  if (perm_out)
    for (int i = 0; i < pnv; ++i) perm_out[i] = perm[i];
  return (int)c.size() == 0 ? 1 : 0;
}
