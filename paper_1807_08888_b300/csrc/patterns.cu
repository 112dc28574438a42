// Top-k frequent patterns by minimum image-based support: Algorithm 2 (Section 3.3) with the
// pattern-mining user functions of Section 4.2 (Listing 2).
//
//   key(s)       = the pattern of s (connected, vertex-labelled, edge-unlabelled, <= 6 vertices)
//   f(S)         = MNI support: min over pattern vertices i of |D_i|, D_i = data vertices that
//                  some embedding maps i to (Section 2; automorphic embeddings included)
//   relevant(S)  = edgeCount == M;  expandable(s, d) = edgeCount < M
//   priority(S)  = (edgeCount, f);  dominated(S, O) = f(S) < f(O) (strict), O = k-th in R
//
// The groups of Algorithm 2 are kept as patterns with their domains instead of member lists:
// the paper's aggregation over members (Listing 2) yields the same f.  The lattice walk (a
// priority queue of a few hundred patterns, canonical codes, duplicate removal) runs on the
// host; every pass over the data graph runs in kernels:
//   * k_one_edge_support: for every vertex u and label l, whether u has a neighbour of label l
//     (non-empty label segment) -> exact supports and domains of all 1-edge patterns;
//   * k_mni_exist: one warp per (pattern, pattern vertex i, candidate u); skipped when u is
//     already in D_i; otherwise a depth-first search for an embedding with i -> u along a
//     breadth-first order from i (candidates from label segments, 32 per step, ballot), with
//     every candidate restricted to the parent pattern's domain (anti-monotonicity: an
//     embedding of the child restricted to the parent is an embedding of the parent).  A found
//     embedding sets the bits of every pattern vertex's image (harvesting);
//   * k_popc: |D_i| by popcount.
// Children whose support is already bounded below tau by a known sub-pattern (the 1-edge
// pattern of the added edge, or the parent) are pruned without a search.
#include <algorithm>
#include <climits>
#include <cstring>
#include <map>
#include <queue>
#include <set>
#include <vector>

#include "nuri_internal.cuh"
#include "topk_common.cuh"

namespace nuri {
namespace {

constexpr int PV = 6;  // pattern vertices (M <= 5 edges)

// ---- host pattern ------------------------------------------------------------------------
struct Pat {
  int nv = 0;
  int lab[PV] = {};
  uint8_t adj[PV] = {};  // adjacency bit masks
  int edges() const {
    int c = 0;
    for (int i = 0; i < nv; ++i) c += __builtin_popcount(adj[i]);
    return c / 2;
  }
};

typedef std::vector<int> Code;

// Canonical code: the smallest [nv, labels in order, upper-triangle adjacency bits row-major]
// over all vertex orders.  Only orders with non-decreasing labels can be smallest, so the
// search enumerates orders inside each block of equal labels.
Code canonical(const Pat& p, int* perm_out) {
  int idx[PV];
  for (int i = 0; i < p.nv; ++i) idx[i] = i;
  std::sort(idx, idx + p.nv, [&](int a, int b) { return p.lab[a] < p.lab[b]; });
  Code best;
  int bestperm[PV] = {};
  int perm[PV];
  // enumerate permutations within equal-label blocks
  std::vector<std::pair<int, int>> blocks;
  for (int i = 0; i < p.nv;) {
    int j = i;
    while (j < p.nv && p.lab[idx[j]] == p.lab[idx[i]]) ++j;
    blocks.push_back({i, j});
    i = j;
  }
  for (int i = 0; i < p.nv; ++i) perm[i] = idx[i];
  // iterate over the product of block permutations
  std::vector<std::vector<int>> bp(blocks.size());
  for (size_t b = 0; b < blocks.size(); ++b)
    for (int i = blocks[b].first; i < blocks[b].second; ++i) bp[b].push_back(idx[i]);
  for (auto& v : bp) std::sort(v.begin(), v.end());
  while (true) {
    int pos = 0;
    for (auto& v : bp)
      for (int x : v) perm[pos++] = x;
    Code c;
    c.reserve(1 + p.nv + p.nv * (p.nv - 1) / 2);
    c.push_back(p.nv);
    for (int i = 0; i < p.nv; ++i) c.push_back(p.lab[perm[i]]);
    for (int a = 0; a < p.nv; ++a)
      for (int b = a + 1; b < p.nv; ++b) c.push_back((p.adj[perm[a]] >> perm[b]) & 1);
    if (best.empty() || c < best) {
      best = c;
      for (int i = 0; i < p.nv; ++i) bestperm[i] = perm[i];
    }
    // next combination of block permutations
    size_t b = 0;
    for (; b < bp.size(); ++b) {
      if (std::next_permutation(bp[b].begin(), bp[b].end())) break;
    }
    if (b == bp.size()) break;
  }
  if (perm_out)
    for (int i = 0; i < p.nv; ++i) perm_out[i] = bestperm[i];
  return best;
}

Pat relabel(const Pat& p, const int* perm) {  // vertex x of the result = vertex perm[x] of p
  Pat q;
  q.nv = p.nv;
  int inv[PV];
  for (int x = 0; x < p.nv; ++x) inv[perm[x]] = x;
  for (int x = 0; x < p.nv; ++x) {
    q.lab[x] = p.lab[perm[x]];
    uint8_t m = 0;
    for (int y = 0; y < p.nv; ++y)
      if ((p.adj[perm[x]] >> y) & 1) m |= (uint8_t)(1u << inv[y]);
    q.adj[x] = m;
  }
  return q;
}

// ---- device pattern ------------------------------------------------------------------------
struct PatDev {
  int32_t nv;
  int32_t lab[PV];
  int32_t order[PV][PV];  // breadth-first order from each start vertex
  int32_t ppos[PV][PV];   // position of the tree parent in that order
  uint32_t back[PV][PV];  // earlier positions adjacent, parent excluded
  int32_t filt[PV];       // bitmap slot restricting the candidates of vertex j (-1: none)
  int32_t dom;            // first bitmap slot of this pattern's domains (nv slots)
};

struct MniCtx {
  DevGraph g;
  const PatDev* pats;
  uint32_t* bits;        // bitmap slots, words_per_slot words each
  int64_t words;         // words per slot
  unsigned long long* work;
  unsigned long long* counters;  // [0] searches, [1] found, [2] skipped, [3] bytes
  const uint64_t* deadline;      // global timer value after which the search stops
  int32_t* err;                  // bit 2: time budget exhausted
};

__device__ __forceinline__ bool bit_get(const uint32_t* b, int32_t u) {
  return (__ldg(b + (u >> 5)) >> (u & 31)) & 1u;
}

__device__ __forceinline__ bool row_has(const DevGraph& g, int32_t a, int32_t b) {
  int64_t ra = g.off[a], ea = g.off[a + 1], rb = g.off[b], eb = g.off[b + 1];
  int32_t x = b;
  if (eb - rb < ea - ra) {
    ra = rb;
    ea = eb;
    x = a;
  }
  int64_t lo = ra, hi = ea;
  while (lo < hi) {
    int64_t mid = (lo + hi) >> 1;
    if (__ldg(g.adj + mid) < x) lo = mid + 1;
    else hi = mid;
  }
  return lo < ea && __ldg(g.adj + lo) == x;
}

// 1-edge supports: has[u * L + l] = u has a neighbour of label l; counts[a * L + b] += 1 for
// every vertex u of label a with a neighbour of label b; domain bitmaps of (a, b) built later.
__global__ void k_one_edge_support(DevGraph g, unsigned long long* counts) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < (int64_t)g.n * g.L;
       t += (int64_t)gridDim.x * blockDim.x) {
    int64_t u = t / g.L;
    int l = (int)(t % g.L);
    if (g.lsoff[t + 1] > g.lsoff[t]) atomicAdd(counts + (int64_t)g.labels[u] * g.L + l, 1ull);
  }
}

// domain of a 1-edge pattern vertex: label a with a neighbour of label b
__global__ void k_one_edge_domain(DevGraph g, int32_t a, int32_t b, uint32_t* bits) {
  for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < g.n;
       u += (int64_t)gridDim.x * blockDim.x) {
    if (g.labels[u] != a) continue;
    int64_t t = u * g.L + b;
    if (g.lsoff[t + 1] > g.lsoff[t]) atomicOr(bits + (u >> 5), 1u << (u & 31));
  }
}

struct Item {
  int32_t pat;   // pattern slot in the batch
  int32_t i;     // start vertex
  int32_t u;     // candidate data vertex
};

__global__ void __launch_bounds__(256) k_mni_exist(MniCtx cx, const Item* __restrict__ items,
                                                   int64_t nitems) {
  const int lane = threadIdx.x & 31;
  const unsigned FULL = 0xffffffffu;
  const DevGraph& g = cx.g;
  unsigned long long n_search = 0, n_found = 0, n_skip = 0, n_bytes = 0;
  while (true) {
    int64_t it = 0;
    if (lane == 0) {
      it = (int64_t)atomicAdd(cx.work, 1ull);
      if (it < nitems && global_ns() > *(const volatile uint64_t*)cx.deadline) {
        atomicOr(cx.err, 4);
        it = nitems;
      }
    }
    it = __shfl_sync(FULL, it, 0);
    if (it >= nitems) break;
    Item I = items[it];
    const PatDev& P = cx.pats[I.pat];
    uint32_t* Di = cx.bits + (int64_t)(P.dom + I.i) * cx.words;
    // other warps set domain bits meanwhile: one reading for the warp
    if ((warp_load(Di + (I.u >> 5)) >> (I.u & 31)) & 1u) {
      if (lane == 0) ++n_skip;
      continue;
    }
    if (lane == 0) ++n_search;
    const int nv = P.nv;
    const int32_t* ord = P.order[I.i];
    int32_t mu[PV];      // data vertex per position
    int64_t pos[PV], end[PV], base[PV];
    unsigned mask[PV];
    mu[0] = I.u;
    bool found = nv == 1;
    int lev = 1;
    if (!found) {
      int32_t a = mu[P.ppos[I.i][1]];
      int64_t so = (int64_t)a * g.L + P.lab[ord[1]];
      pos[1] = g.lsoff[so];
      end[1] = g.lsoff[so + 1];
      mask[1] = 0;
    }
    unsigned steps = 0;
    bool stop = false;
    while (!found && lev >= 1) {
      if (mask[lev] == 0) {
        if (pos[lev] >= end[lev]) {
          --lev;
          continue;
        }
        if ((++steps & 255) == 0 && warp_past(cx.deadline)) {
          if (lane == 0) atomicOr(cx.err, 4);
          stop = true;
          break;
        }
        int64_t t = pos[lev] + lane;
        bool valid = t < end[lev];
        int32_t x = valid ? __ldg(g.lseg_d + t).x : -1;
        if (valid)
          for (int a = 0; a < lev; ++a)
            if (mu[a] == x) valid = false;
        int j = ord[lev];
        if (valid && P.filt[j] >= 0) valid = bit_get(cx.bits + (int64_t)P.filt[j] * cx.words, x);
        if (valid) {
          uint32_t m = P.back[I.i][lev];
          while (m && valid) {
            int a = __ffs(m) - 1;
            m &= m - 1;
            valid = row_has(g, mu[a], x);
          }
        }
        unsigned vm = __ballot_sync(FULL, valid);
        if (lane == 0) n_bytes += 8ull * (uint64_t)(end[lev] - pos[lev] < 32 ? end[lev] - pos[lev] : 32);
        base[lev] = pos[lev];
        pos[lev] += 32;
        mask[lev] = vm;
        if (vm && lev == nv - 1) {
          int b = __ffs(vm) - 1;
          mu[lev] = __ldg(g.lseg_d + base[lev] + b).x;
          found = true;
          break;
        }
        continue;
      }
      int b = __ffs(mask[lev]) - 1;
      mask[lev] &= mask[lev] - 1;
      mu[lev] = __ldg(g.lseg_d + base[lev] + b).x;
      ++lev;
      int32_t a = mu[P.ppos[I.i][lev]];
      int64_t so = (int64_t)a * g.L + P.lab[ord[lev]];
      pos[lev] = g.lsoff[so];
      end[lev] = g.lsoff[so + 1];
      mask[lev] = 0;
    }
    if (stop) found = false;
    if (found && lane < nv) {
      // harvest: every pattern vertex's image joins its domain
      int32_t v = mu[lane];
      int j = ord[lane];
      uint32_t* Dj = cx.bits + (int64_t)(P.dom + j) * cx.words;
      atomicOr(Dj + (v >> 5), 1u << (v & 31));
    }
    if (found && lane == 0) ++n_found;
  }
  if (lane == 0) {
    atomicAdd(cx.counters + 0, n_search);
    atomicAdd(cx.counters + 1, n_found);
    atomicAdd(cx.counters + 2, n_skip);
    atomicAdd(cx.counters + 3, n_bytes);
  }
}

// candidate items: every set bit of a bitmap (or every vertex of a label) for (pat, i)
__global__ void k_items_from_bits(const uint32_t* bits, int64_t words, int32_t pat, int32_t i,
                                  Item* out, unsigned long long* cnt) {
  for (int64_t w = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; w < words;
       w += (int64_t)gridDim.x * blockDim.x) {
    uint32_t x = bits[w];
    if (!x) continue;
    unsigned long long base = atomicAdd(cnt, (unsigned long long)__popc(x));
    while (x) {
      int b = __ffs(x) - 1;
      x &= x - 1;
      out[base++] = Item{pat, i, (int32_t)(w * 32 + b)};
    }
  }
}

__global__ void k_items_from_label(DevGraph g, int32_t lab, int32_t pat, int32_t i, Item* out,
                                   unsigned long long* cnt) {
  int64_t b = g.lab_off[lab], e = g.lab_off[lab + 1];
  for (int64_t t = b + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < e;
       t += (int64_t)gridDim.x * blockDim.x) {
    unsigned long long p = atomicAdd(cnt, 1ull);
    out[p] = Item{pat, i, g.lab_vert[t]};
  }
}

__global__ void k_popc(const uint32_t* bits, int64_t words, int32_t nslots, const int32_t* slot,
                       unsigned long long* out) {
  // one block per requested slot
  for (int s = blockIdx.x; s < nslots; s += gridDim.x) {
    const uint32_t* b = bits + (int64_t)slot[s] * words;
    unsigned long long c = 0;
    for (int64_t w = threadIdx.x; w < words; w += blockDim.x) c += __popc(b[w]);
    for (int o = 16; o; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    __shared__ unsigned long long red[32];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
      unsigned long long t = 0;
      for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += red[i];
      out[s] = t;
    }
    __syncthreads();
  }
}

inline int gridp(int64_t n) {
  int64_t b = (n + 255) / 256;
  return (int)std::max<int64_t>(1, std::min<int64_t>(b, 1 << 20));
}

// ---- bitmap pool on the device ------------------------------------------------------------
struct Pool {
  DBuf<uint32_t> mem;
  int64_t words = 0;
  int32_t cap = 0;
  std::vector<int32_t> free_slots;
  cudaStream_t s;
  void init(int64_t w, int32_t c, cudaStream_t st) {
    s = st;
    words = w;
    cap = c;
    mem.alloc((int64_t)c * w, st);
    free_slots.clear();
    for (int i = c - 1; i >= 0; --i) free_slots.push_back(i);
  }
  int32_t take() {
    if (free_slots.empty()) grow();
    int32_t x = free_slots.back();
    free_slots.pop_back();
    NURI_CUDA(cudaMemsetAsync(mem.p + (int64_t)x * words, 0, sizeof(uint32_t) * words, s));
    return x;
  }
  void give(int32_t x) { free_slots.push_back(x); }
  void grow() {
    int32_t nc = std::max(cap * 2, 16);
    DBuf<uint32_t> nm;
    nm.alloc((int64_t)nc * words, s);
    if (cap) NURI_CUDA(cudaMemcpyAsync(nm.p, mem.p, sizeof(uint32_t) * cap * words, cudaMemcpyDeviceToDevice, s));
    mem = std::move(nm);
    for (int i = nc - 1; i >= cap; --i) free_slots.push_back(i);
    cap = nc;
  }
};

struct Group {
  Pat p;
  Code code;
  int64_t f;
  int32_t dom[PV];  // bitmap slots of the domains (-1: not resident)
};

void fill_orders(const Pat& p, PatDev* d) {
  d->nv = p.nv;
  for (int i = 0; i < p.nv; ++i) d->lab[i] = p.lab[i];
  for (int s0 = 0; s0 < p.nv; ++s0) {
    int order[PV], pos[PV], par[PV];
    for (int i = 0; i < p.nv; ++i) pos[i] = -1, par[i] = -1;
    int head = 0, tail = 0;
    order[tail++] = s0;
    pos[s0] = 0;
    while (head < tail) {
      int a = order[head++];
      for (int b = 0; b < p.nv; ++b)
        if (((p.adj[a] >> b) & 1) && pos[b] < 0) {
          pos[b] = tail;
          par[b] = a;
          order[tail++] = b;
        }
    }
    for (int t = 0; t < p.nv; ++t) {
      int j = order[t];
      d->order[s0][t] = j;
      d->ppos[s0][t] = t == 0 ? -1 : pos[par[j]];
      uint32_t bk = 0;
      for (int u = 0; u < t; ++u)
        if (((p.adj[j] >> order[u]) & 1) && u != d->ppos[s0][t]) bk |= 1u << u;
      d->back[s0][t] = bk;
    }
  }
}

}  // namespace

void topk_patterns(nuri_graph* G, int32_t M, int32_t k, uint32_t flags, cudaStream_t s,
                   nuri_result** out) {
  const DevGraph& g = G->d;
  DevTimer timer(s);
  const bool keep_ties = flags & NURI_KEEP_TIES;
  const int L = g.L;
  int64_t launches = 0;
  nuri_stats stats;
  memset(&stats, 0, sizeof(stats));
  const int64_t words = ((int64_t)g.n + 31) / 32;

  // 1-edge supports
  std::vector<unsigned long long> cnt((size_t)L * L, 0);
  {
    DBuf<unsigned long long> dc;
    dc.alloc((size_t)L * L, s);
    NURI_CUDA(cudaMemsetAsync(dc.p, 0, sizeof(unsigned long long) * L * L, s));
    if (g.n > 0) {
      ++launches;
      k_one_edge_support<<<gridp((int64_t)g.n * L), 256, 0, s>>>(g, dc.p);
    }
    NURI_CUDA(cudaMemcpyAsync(cnt.data(), dc.p, sizeof(unsigned long long) * L * L, cudaMemcpyDeviceToHost, s));
    NURI_CUDA(cudaStreamSynchronize(s));
  }
  auto f1 = [&](int a, int b) -> int64_t {
    if (a == b) return (int64_t)cnt[(size_t)a * L + a];
    return (int64_t)std::min(cnt[(size_t)a * L + b], cnt[(size_t)b * L + a]);
  };

  // result set R (Algorithm 2): entries (f, code, pattern)
  struct REntry {
    int64_t f;
    Code code;
    Pat p;
  };
  std::vector<REntry> R;
  auto kth = [&]() -> int64_t {
    if ((int)R.size() < k) return INT64_MIN;
    std::vector<int64_t> fs;
    for (auto& e : R) fs.push_back(e.f);
    std::nth_element(fs.begin(), fs.begin() + (k - 1), fs.end(), std::greater<int64_t>());
    return fs[k - 1];
  };
  auto offer = [&](const Group& S) {
    int64_t t = kth();
    if (!((int)R.size() < k || S.f >= t)) return;
    R.push_back({S.f, S.code, S.p});
    if ((int)R.size() > k) {
      int64_t t2 = kth();
      R.erase(std::remove_if(R.begin(), R.end(), [&](const REntry& e) { return e.f < t2; }), R.end());
    }
  };

  // priority queue of groups by (edges, f)
  std::vector<Group> store;
  auto cmp = [&](int a, int b) {
    int ea = store[a].p.edges(), eb = store[b].p.edges();
    if (ea != eb) return ea < eb;
    if (store[a].f != store[b].f) return store[a].f < store[b].f;
    return a > b;
  };
  std::priority_queue<int, std::vector<int>, decltype(cmp)> Q(cmp);
  std::set<Code> constructed;
  Pool pool;
  pool.init(words, 64, s);

  // seeds (Algorithm 2, initialisation): one group per 1-edge pattern present
  for (int a = 0; a < L; ++a)
    for (int b = a; b < L; ++b) {
      int64_t f = f1(a, b);
      if (f <= 0) continue;
      Group S;
      S.p.nv = 2;
      S.p.lab[0] = a;
      S.p.lab[1] = b;
      S.p.adj[0] = 2;
      S.p.adj[1] = 1;
      int perm[PV];
      S.code = canonical(S.p, perm);
      S.p = relabel(S.p, perm);
      S.f = f;
      for (int i = 0; i < PV; ++i) S.dom[i] = -1;
      constructed.insert(S.code);
      store.push_back(S);
      Q.push((int)store.size() - 1);
    }

  DBuf<uint64_t> deadline;
  deadline.alloc(1, s);
  DBuf<int32_t> derr;
  derr.alloc(1, s);
  NURI_CUDA(cudaMemsetAsync(derr.p, 0, 4, s));
  ++launches;
  k_set_deadline<<<1, 32, 0, s>>>(deadline.p, time_budget_ns());
  DBuf<unsigned long long> counters, work, icnt;
  counters.alloc(4, s);
  work.alloc(1, s);
  icnt.alloc(1, s);
  NURI_CUDA(cudaMemsetAsync(counters.p, 0, sizeof(unsigned long long) * 4, s));
  DBuf<Item> items;
  DBuf<PatDev> dpats;
  DBuf<int32_t> dslots;
  DBuf<unsigned long long> dpop;
  cudaEvent_t ev0, ev1;
  NURI_CUDA(cudaEventCreate(&ev0));
  NURI_CUDA(cudaEventCreate(&ev1));
  struct EvGuard {
    cudaEvent_t a, b;
    ~EvGuard() {
      cudaEventDestroy(a);
      cudaEventDestroy(b);
    }
  } evg{ev0, ev1};

  // domains of a 1-edge group
  auto ensure_domains = [&](Group& S) {
    if (S.dom[0] >= 0) return;
    if (S.p.nv == 2 && S.p.edges() == 1) {
      for (int i = 0; i < 2; ++i) {
        S.dom[i] = pool.take();
        ++launches;
        k_one_edge_domain<<<gridp(g.n), 256, 0, s>>>(g, S.p.lab[i], S.p.lab[1 - i],
                                                     pool.mem.p + (int64_t)S.dom[i] * words);
      }
    }
  };

  while (!Q.empty()) {
    int si = Q.top();
    Q.pop();
    Group S = store[si];
    ++stats.dequeued;
    int mS = S.p.edges();
    if (mS == M) offer(S);  // relevant
    int64_t tau = kth();
    bool dominated = (int)R.size() >= k && S.f < tau;
    if (dominated || mS >= M) {
      for (int i = 0; i < PV; ++i)
        if (S.dom[i] >= 0) pool.give(S.dom[i]);
      store[si].dom[0] = -1;
      continue;
    }
    // ---- expand the group: child patterns by one more edge ----
    ensure_domains(S);
    struct Child {
      Pat p;
      Code code;
      int64_t ub;
      int32_t from_parent[PV];  // parent vertex of each child vertex (-1: the new vertex)
    };
    std::vector<Child> kids;
    auto consider = [&](const Pat& c0, const int* parent_of, int la, int lb) {
      int perm[PV];
      Code code = canonical(c0, perm);
      if (constructed.count(code)) return;
      constructed.insert(code);
      ++stats.expansions;
      Child c;
      c.p = relabel(c0, perm);
      c.code = code;
      for (int x = 0; x < c0.nv; ++x) c.from_parent[x] = parent_of[perm[x]];
      c.ub = std::min<int64_t>(S.f, f1(std::min(la, lb), std::max(la, lb)));
      if (c.ub <= 0 || ((int)R.size() >= k && c.ub < tau)) {
        ++stats.pruned;
        return;
      }
      kids.push_back(c);
    };
    for (int i = 0; i < S.p.nv; ++i) {
      if (S.p.nv < PV)
        for (int l = 0; l < L; ++l) {  // forward edge to a new vertex of label l
          Pat c0 = S.p;
          c0.lab[c0.nv] = l;
          c0.adj[i] |= (uint8_t)(1u << c0.nv);
          c0.adj[c0.nv] = (uint8_t)(1u << i);
          c0.nv += 1;
          int parent_of[PV];
          for (int x = 0; x < S.p.nv; ++x) parent_of[x] = x;
          parent_of[S.p.nv] = -1;
          consider(c0, parent_of, S.p.lab[i], l);
        }
      for (int j = i + 1; j < S.p.nv; ++j)  // backward edge between two pattern vertices
        if (!((S.p.adj[i] >> j) & 1)) {
          Pat c0 = S.p;
          c0.adj[i] |= (uint8_t)(1u << j);
          c0.adj[j] |= (uint8_t)(1u << i);
          int parent_of[PV];
          for (int x = 0; x < S.p.nv; ++x) parent_of[x] = x;
          consider(c0, parent_of, S.p.lab[i], S.p.lab[j]);
        }
    }
    if (!kids.empty()) {
      // ---- supports of all children in one launch ----
      std::vector<PatDev> hp(kids.size());
      std::vector<Group> kg(kids.size());
      int64_t nitems_cap = 0;
      for (size_t c = 0; c < kids.size(); ++c) {
        fill_orders(kids[c].p, &hp[c]);
        kg[c].p = kids[c].p;
        kg[c].code = kids[c].code;
        for (int x = 0; x < PV; ++x) {
          kg[c].dom[x] = -1;
          hp[c].filt[x] = -1;
        }
        for (int x = 0; x < kids[c].p.nv; ++x) {
          int pv = kids[c].from_parent[x];
          int lab = kids[c].p.lab[x];
          nitems_cap += pv >= 0 ? g.n : (G->h_lab_off[lab + 1] - G->h_lab_off[lab]);
        }
      }
      // one buffer holds every child's domains (nv slots each) followed by copies of the
      // parent's domains, which restrict the candidates (anti-monotonicity)
      int32_t nslot = 0;
      for (auto& c : kids) nslot += c.p.nv;
      int32_t filt_base = nslot;
      DBuf<uint32_t> allbits;
      allbits.alloc((int64_t)(nslot + S.p.nv) * words, s);
      NURI_CUDA(cudaMemsetAsync(allbits.p, 0, sizeof(uint32_t) * nslot * words, s));
      for (int x = 0; x < S.p.nv; ++x)
        NURI_CUDA(cudaMemcpyAsync(allbits.p + (int64_t)(filt_base + x) * words,
                                  pool.mem.p + (int64_t)S.dom[x] * words,
                                  sizeof(uint32_t) * words, cudaMemcpyDeviceToDevice, s));
      int32_t slot = 0;
      for (size_t c = 0; c < kids.size(); ++c) {
        hp[c].dom = slot;
        for (int x = 0; x < kids[c].p.nv; ++x) {
          int pv = kids[c].from_parent[x];
          hp[c].filt[x] = pv >= 0 ? filt_base + pv : -1;
        }
        slot += kids[c].p.nv;
      }
      dpats.alloc(kids.size(), s);
      NURI_CUDA(cudaMemcpyAsync(dpats.p, hp.data(), sizeof(PatDev) * kids.size(), cudaMemcpyHostToDevice, s));
      if ((int64_t)items.n < nitems_cap) items.alloc(std::max<int64_t>(nitems_cap, 1024), s);
      NURI_CUDA(cudaMemsetAsync(icnt.p, 0, 8, s));
      for (size_t c = 0; c < kids.size(); ++c)
        for (int x = 0; x < kids[c].p.nv; ++x) {
          int pv = kids[c].from_parent[x];
          ++launches;
          if (pv >= 0)
            k_items_from_bits<<<gridp(words), 256, 0, s>>>(
                allbits.p + (int64_t)(filt_base + pv) * words, words, (int32_t)c, x, items.p, icnt.p);
          else
            k_items_from_label<<<gridp(G->h_lab_off[kids[c].p.lab[x] + 1] - G->h_lab_off[kids[c].p.lab[x]]), 256, 0, s>>>(
                g, kids[c].p.lab[x], (int32_t)c, x, items.p, icnt.p);
        }
      unsigned long long nitems = 0;
      NURI_CUDA(cudaMemcpyAsync(&nitems, icnt.p, 8, cudaMemcpyDeviceToHost, s));
      NURI_CUDA(cudaStreamSynchronize(s));
      MniCtx cx;
      cx.g = g;
      cx.pats = dpats.p;
      cx.bits = allbits.p;
      cx.words = words;
      cx.work = work.p;
      cx.counters = counters.p;
      cx.deadline = deadline.p;
      cx.err = derr.p;
      NURI_CUDA(cudaMemsetAsync(work.p, 0, 8, s));
      NURI_CUDA(cudaEventRecord(ev0, s));
      if (nitems > 0) {
        ++launches;
        k_mni_exist<<<sm_count() * 8, 256, 0, s>>>(cx, items.p, (int64_t)nitems);
      }
      NURI_CUDA(cudaEventRecord(ev1, s));
      // domain sizes
      std::vector<int32_t> slots(nslot);
      for (int i = 0; i < nslot; ++i) slots[i] = i;
      dslots.alloc(std::max(nslot, 1), s);
      dpop.alloc(std::max(nslot, 1), s);
      NURI_CUDA(cudaMemcpyAsync(dslots.p, slots.data(), sizeof(int32_t) * nslot, cudaMemcpyHostToDevice, s));
      ++launches;
      k_popc<<<std::min(nslot, 4096), 256, 0, s>>>(allbits.p, words, nslot, dslots.p, dpop.p);
      std::vector<unsigned long long> pop(nslot);
      NURI_CUDA(cudaMemcpyAsync(pop.data(), dpop.p, sizeof(unsigned long long) * nslot, cudaMemcpyDeviceToHost, s));
      int32_t herr = 0;
      NURI_CUDA(cudaMemcpyAsync(&herr, derr.p, 4, cudaMemcpyDeviceToHost, s));
      NURI_CUDA(cudaStreamSynchronize(s));
      if (herr & 4) NURI_FAIL(NURI_ERR_TIMEOUT, "nuri_topk_patterns: time budget exhausted");
      {
        float ms = 0.f;
        NURI_CUDA(cudaEventElapsedTime(&ms, ev0, ev1));
        stats.expand_ms += ms;
        stats.expand_launches += 1;
      }
      ++stats.rounds;
      // move the children's domains into the pool (kept while they wait in the queue)
      for (size_t c = 0; c < kids.size(); ++c) {
        int64_t f = INT64_MAX;
        for (int x = 0; x < kids[c].p.nv; ++x) f = std::min<int64_t>(f, (int64_t)pop[hp[c].dom + x]);
        kg[c].f = f;
        bool keep = f > 0 && ((int)R.size() < k || f >= kth());
        if (keep && kids[c].p.edges() < M)
          for (int x = 0; x < kids[c].p.nv; ++x) {
            kg[c].dom[x] = pool.take();
            NURI_CUDA(cudaMemcpyAsync(pool.mem.p + (int64_t)kg[c].dom[x] * words,
                                      allbits.p + (int64_t)(hp[c].dom + x) * words,
                                      sizeof(uint32_t) * words, cudaMemcpyDeviceToDevice, s));
          }
        if (!keep) {
          ++stats.pruned;
          continue;
        }
        store.push_back(kg[c]);
        Q.push((int)store.size() - 1);  // enqueue the child group
      }
      NURI_CUDA(cudaStreamSynchronize(s));
    }
    for (int i = 0; i < PV; ++i)
      if (S.dom[i] >= 0) pool.give(S.dom[i]);
    store[si].dom[0] = -1;
  }

  // ---- results: (f desc, canonical code asc), first k (or every tie) ----
  std::sort(R.begin(), R.end(), [](const REntry& a, const REntry& b) {
    if (a.f != b.f) return a.f > b.f;
    return a.code < b.code;
  });
  int32_t count = (int32_t)R.size();
  if (!keep_ties) count = std::min(count, k);
  int64_t nverts = 0, nedges = 0;
  for (int i = 0; i < count; ++i) {
    nverts += R[i].p.nv;
    nedges += R[i].p.edges();
  }
  nuri_result* r = new_result(2, count, nverts, nedges, true);
  int64_t pv = 0, pe = 0;
  for (int i = 0; i < count; ++i) {
    r->score[i] = R[i].f;
    r->vert_off[i] = (int32_t)pv;
    r->edge_off[i] = (int32_t)pe;
    const Pat& p = R[i].p;
    for (int x = 0; x < p.nv; ++x) {
      r->verts[pv] = x;
      r->labels[pv] = p.lab[x];
      ++pv;
    }
    for (int a = 0; a < p.nv; ++a)
      for (int b = a + 1; b < p.nv; ++b)
        if ((p.adj[a] >> b) & 1) {
          r->edges[2 * pe] = a;
          r->edges[2 * pe + 1] = b;
          ++pe;
        }
  }
  r->vert_off[count] = (int32_t)pv;
  r->edge_off[count] = (int32_t)pe;
  unsigned long long hc[4];
  NURI_CUDA(cudaMemcpyAsync(hc, counters.p, sizeof(hc), cudaMemcpyDeviceToHost, s));
  NURI_CUDA(cudaStreamSynchronize(s));
  stats.results_stored = (int64_t)R.size();
  stats.threshold = kth();
  stats.adj_bytes = (int64_t)hc[3];
  stats.device_ms = timer.stop();
  stats.launches = launches;
  r->stats = stats;
  *out = r;
}

}  // namespace nuri
