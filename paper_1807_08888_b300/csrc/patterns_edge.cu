// Top-k frequent patterns by edge-oriented exhaustive expansion: the other way Section 2 grows
// subgraphs (one-edge subgraphs, then one edge at a time), the way Arabesque mines patterns
// (Section 2.2): every connected subgraph with M edges is enumerated once, grouped by its
// pattern, and each pattern's minimum image-based support is taken over all its embeddings.
// Nothing is pruned: it is the ablation beside Algorithm 2 (the same call without
// NURI_PATTERNS_EDGE_ORIENTED), which never expands patterns that cannot reach the k-th
// support.  Both return the same rows.
//
// GPU organisation:
//   * the undirected edges {a, b} (a < b) numbered in CSR order; eid[t] = the number of the
//     edge of CSR entry t (either direction);
//   * k_esu: one warp per seed edge e0 (dynamic).  ESU on the line graph enumerates every
//     connected edge set once, from its smallest edge: a node holds its edges S and an
//     extension list of edges after e0 adjacent to S; the child through the list's i-th edge w
//     keeps the list's tail after w and adds the edges after e0 at w's new endpoint whose other
//     endpoint is new too (edges at an old vertex are adjacent to S already: in the list or
//     passed over).  Lists live in per-warp global scratch; the lanes build them (ballot) and
//     take the leaves (S plus one listed edge) one each;
//   * per leaf: its canonical code (the smallest [n, labels, upper-triangle bits] over vertex
//     orders with non-decreasing labels) -- pass 1 writes the codes, which sorted and made
//     unique are the patterns; pass 2 looks a leaf's code up and sets, for every vertex order
//     reaching the smallest code (automorphic embeddings included), the domain bit of each
//     image vertex;
//   * MNI = min over pattern vertices of the domain's popcount; rows ordered by (MNI desc,
//     code asc) with radix passes.
#include <cub/cub.cuh>

#include <algorithm>
#include <cstring>
#include <vector>

#include "nuri_internal.cuh"
#include "topk_common.cuh"

namespace nuri {
namespace {

constexpr int EPV = 6;            // pattern vertices (M <= 5 edges)
constexpr int EXTCAP = 4096;      // extension-list entries per level and warp
constexpr int ESU_WARPS = 8;      // warps per block

struct EsuCtx {
  DevGraph g;
  const int32_t* eu;   // [m] edge endpoints, eu < ev
  const int32_t* ev;
  const int64_t* eid;  // [nnz] edge number of every CSR entry
  int64_t m;
  int32_t M;
  int32_t pass;        // 1: write codes, 2: set domain bits
  int32_t* scratch;    // per warp: M levels of EXTCAP entries
  unsigned long long* table;  // pass 1: hash set of the patterns' packed codes
  int64_t table_mask;
  int32_t lb;                 // bits per label in a packed code
  const unsigned long long* pat;  // pass 2: the patterns' packed codes, sorted
  int64_t npat;
  uint32_t* dom;       // pass 2: [npat][EPV][words]
  int64_t words;
  unsigned long long* work;
  unsigned long long* nodes;  // ESU nodes visited (every edge set grown, leaves included)
  unsigned long long* leaves; // embeddings (connected M-edge subgraphs)
  int32_t* err;        // bit 0: an extension list above EXTCAP; bit 2: time budget exhausted;
                       // bit 3: the pattern hash set is full
  const uint64_t* deadline;
};

__device__ __forceinline__ int64_t row_pos(const DevGraph& g, int32_t a, int32_t b) {
  int64_t lo = g.off[a], hi = g.off[a + 1];
  const int64_t end = hi;
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (__ldg(g.adj + mid) < b) lo = mid + 1;
    else hi = mid;
  }
  return lo < end && __ldg(g.adj + lo) == b ? lo : -1;
}

// keep[t] = 1 when CSR entry t is the (a < b) direction of its edge
__global__ void k_edge_flags(DevGraph g, int64_t* __restrict__ keep) {
  const int lane = threadIdx.x & 31;
  for (int64_t v = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; v < g.n;
       v += ((int64_t)gridDim.x * blockDim.x) >> 5)
    for (int64_t t = g.off[v] + lane; t < g.off[v + 1]; t += 32) keep[t] = g.adj[t] > v ? 1 : 0;
}

// with pos = exclusive prefix of keep: the edge list, and eid of every entry (the mirror entry
// of a > b found by binary search)
__global__ void k_edge_ids(DevGraph g, const int64_t* __restrict__ pos, int32_t* __restrict__ eu,
                           int32_t* __restrict__ ev, int64_t* __restrict__ eid) {
  const int lane = threadIdx.x & 31;
  for (int64_t v = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; v < g.n;
       v += ((int64_t)gridDim.x * blockDim.x) >> 5)
    for (int64_t t = g.off[v] + lane; t < g.off[v + 1]; t += 32) {
      const int32_t b = g.adj[t];
      if (b > v) {
        eu[pos[t]] = (int32_t)v;
        ev[pos[t]] = b;
        eid[t] = pos[t];
      } else {
        const int64_t m = row_pos(g, b, (int32_t)v);  // exists: the CSR is symmetric
        eid[t] = m >= 0 ? pos[m] : -1;
      }
    }
}

// next permutation of a[lo, hi) (ascending order), false after the last one
__device__ bool next_perm(int* a, int lo, int hi) {
  int i = hi - 2;
  while (i >= lo && a[i] >= a[i + 1]) --i;
  if (i < lo) {
    for (int l = lo, r = hi - 1; l < r; ++l, --r) {
      const int t = a[l];
      a[l] = a[r];
      a[r] = t;
    }
    return false;
  }
  int j = hi - 1;
  while (a[j] <= a[i]) --j;
  int t = a[i];
  a[i] = a[j];
  a[j] = t;
  for (int l = i + 1, r = hi - 1; l < r; ++l, --r) {
    t = a[l];
    a[l] = a[r];
    a[r] = t;
  }
  return true;
}

// Canonical code of a labelled graph on nv <= 6 vertices (adjacency masks adjm): hi = nv and
// the labels in non-decreasing order, lo = the upper-triangle bits row-major, first bit most
// significant, smallest over the orders within blocks of equal labels.  With visit set, calls
// visit(order) for every order reaching the smallest lo (order[pos] = vertex at position pos).
template <class F>
__device__ void canon_code(int nv, const int* lab, const uint8_t* adjm, unsigned long long* hi,
                           unsigned long long* lo, bool second_sweep, F&& visit) {
  int ord[EPV];
  for (int i = 0; i < nv; ++i) ord[i] = i;
  for (int i = 1; i < nv; ++i) {  // stable insertion sort by label
    const int x = ord[i];
    int j = i - 1;
    while (j >= 0 && lab[ord[j]] > lab[x]) {
      ord[j + 1] = ord[j];
      --j;
    }
    ord[j + 1] = x;
  }
  unsigned long long h = (unsigned long long)nv << 48;
  for (int i = 0; i < nv; ++i) h |= (unsigned long long)(lab[ord[i]] & 0xff) << (40 - 8 * i);
  int bstart[EPV + 1], nb = 0;
  for (int i = 0; i < nv; ++i)
    if (i == 0 || lab[ord[i]] != lab[ord[i - 1]]) bstart[nb++] = i;
  bstart[nb] = nv;
  const int ntri = nv * (nv - 1) / 2;
  auto code_of = [&](const int* o) {
    unsigned long long c = 0;
    int idx = 0;
    for (int a = 0; a < nv; ++a)
      for (int b = a + 1; b < nv; ++b, ++idx)
        if ((adjm[o[a]] >> o[b]) & 1) c |= 1ull << (ntri - 1 - idx);
    return c;
  };
  unsigned long long best = ~0ull;
  for (int sweep = 0; sweep < (second_sweep ? 2 : 1); ++sweep) {
    int o[EPV];
    for (int i = 0; i < nv; ++i) o[i] = ord[i];
    // blocks start sorted by vertex index (the first permutation of each)
    for (int b = 0; b < nb; ++b)
      for (int i = bstart[b] + 1; i < bstart[b + 1]; ++i) {
        const int x = o[i];
        int j = i - 1;
        while (j >= bstart[b] && o[j] > x) {
          o[j + 1] = o[j];
          --j;
        }
        o[j + 1] = x;
      }
    while (true) {
      const unsigned long long c = code_of(o);
      if (sweep == 0) {
        if (c < best) best = c;
      } else if (c == best) {
        visit(o);
      }
      int b = 0;
      for (; b < nb; ++b)
        if (next_perm(o, bstart[b], bstart[b + 1])) break;
      if (b == nb) break;
    }
  }
  *hi = h;
  *lo = best;
}

// The code packed into 64 bits in the same order: nv (3 bits), the labels (lb bits each, in
// order, from bit 60 down) and the upper-triangle bits (the low 15).
__device__ __forceinline__ unsigned long long pack_code(unsigned long long hi,
                                                        unsigned long long lo, int lb) {
  const int nv = (int)(hi >> 48);
  unsigned long long key = (unsigned long long)nv << 61;
  for (int i = 0; i < nv; ++i)
    key |= ((hi >> (40 - 8 * i)) & 0xffull) << (61 - lb * (i + 1));
  return key | lo;
}

__device__ __forceinline__ unsigned long long mix64(unsigned long long x) {
  x ^= x >> 30;
  x *= 0xbf58476d1ce4e5b9ull;
  x ^= x >> 27;
  x *= 0x94d049bb133111ebull;
  return x ^ (x >> 31);
}

// One leaf: the node's edges (vertex indices sa/sb into vs) plus edge w.
__device__ void esu_leaf(const EsuCtx& cx, const int32_t* vs, int nvs, const int8_t* sa,
                         const int8_t* sb, int ns, int64_t w) {
  int32_t v[EPV];
  int nv = nvs;
  for (int i = 0; i < nvs; ++i) v[i] = vs[i];
  const int32_t a = cx.eu[w], b = cx.ev[w];
  int ia = -1, ib = -1;
  for (int i = 0; i < nvs; ++i) {
    if (v[i] == a) ia = i;
    if (v[i] == b) ib = i;
  }
  // a listed edge touches the node, so at most one endpoint is new (both only for a seed)
  if (nv + (ia < 0) + (ib < 0) > EPV) return;
  if (ia < 0) {
    ia = nv;
    v[nv++] = a;
  }
  if (ib < 0) {
    ib = nv;
    v[nv++] = b;
  }
  uint8_t adjm[EPV] = {0, 0, 0, 0, 0, 0};
  for (int e = 0; e < ns; ++e) {
    adjm[sa[e]] |= 1 << sb[e];
    adjm[sb[e]] |= 1 << sa[e];
  }
  adjm[ia] |= 1 << ib;
  adjm[ib] |= 1 << ia;
  int lab[EPV];
  for (int i = 0; i < nv; ++i) lab[i] = __ldg(cx.g.labels + v[i]);
  unsigned long long hi = 0, lo = 0;
  canon_code(nv, lab, adjm, &hi, &lo, false, [](const int*) {});
  const unsigned long long key = pack_code(hi, lo, cx.lb);
  if (cx.pass == 1) {
    // into the hash set (a plain read first: most leaves find their pattern there)
    int64_t h = (int64_t)(mix64(key) & (unsigned long long)cx.table_mask);
    for (int64_t probe = 0; probe <= cx.table_mask; ++probe) {
      const unsigned long long cur = *(volatile unsigned long long*)(cx.table + h);
      if (cur == key) return;
      if (cur == ~0ull) {
        const unsigned long long prev = atomicCAS(cx.table + h, ~0ull, key);
        if (prev == ~0ull || prev == key) return;
      }
      h = (h + 1) & cx.table_mask;
    }
    atomicOr(cx.err, 8);
    return;
  }
  // the pattern's number: binary search in the sorted codes
  int64_t l = 0, r = cx.npat;
  while (l < r) {
    const int64_t mid = (l + r) >> 1;
    if (cx.pat[mid] < key) l = mid + 1;
    else r = mid;
  }
  if (l >= cx.npat || cx.pat[l] != key) return;  // cannot happen
  uint32_t* D = cx.dom + l * EPV * cx.words;
  canon_code(nv, lab, adjm, &hi, &lo, true, [&](const int* o) {
    for (int pos = 0; pos < nv; ++pos) {
      const int32_t x = v[o[pos]];
      atomicOr(D + pos * cx.words + (x >> 5), 1u << (x & 31));
    }
  });
}

__global__ void __launch_bounds__(ESU_WARPS * 32) k_esu(EsuCtx cx) {
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int64_t gwarp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  int32_t* ext = cx.scratch + gwarp * (int64_t)cx.M * EXTCAP;  // level d: ext + d * EXTCAP
  const DevGraph& g = cx.g;
  unsigned long long my_nodes = 0, my_leaves = 0;
  while (true) {
    long long e0 = 0;
    if (lane == 0) {
      e0 = (long long)atomicAdd(cx.work, 1ull);
      if (e0 < cx.m && global_ns() > *(const volatile uint64_t*)cx.deadline) {
        atomicOr(cx.err, 4);
        e0 = cx.m;
      }
    }
    e0 = __shfl_sync(FULL, e0, 0);
    if (e0 >= cx.m) break;
    // the node: vertices vs, edges (sa, sb) as vertex indices; identical in every lane
    int32_t vs[EPV];
    int8_t sa[5], sb[5];
    int nvs = 2, ns = 1;
    vs[0] = cx.eu[e0];
    vs[1] = cx.ev[e0];
    sa[0] = 0;
    sb[0] = 1;
    if (cx.M == 1) {
      if (lane == 0) {
        ++my_nodes;
        ++my_leaves;
        // the seed itself is the leaf: S = {} plus e0
        esu_leaf(cx, vs, 0, sa, sb, 0, e0);
      }
      continue;
    }
    // level 0 list: edges after e0 at either endpoint
    int n0 = 0;
    bool over = false;
    for (int side = 0; side < 2; ++side) {
      const int32_t x = vs[side];
      for (int64_t b0 = g.off[x]; b0 < g.off[x + 1]; b0 += 32) {
        const int64_t t = b0 + lane;
        const int64_t id = t < g.off[x + 1] ? __ldg(cx.eid + t) : -1;
        const bool keep = id > e0;
        const unsigned bal = __ballot_sync(FULL, keep);
        const int at = n0 + __popc(bal & ((1u << lane) - 1));
        if (keep && at < EXTCAP) ext[at] = (int32_t)id;
        n0 += __popc(bal);
      }
    }
    __syncwarp();
    if (n0 > EXTCAP) over = true;
    if (lane == 0) ++my_nodes;  // the seed
    // depth-first over levels 0 .. M-2 (a node at level d has d + 1 edges and nv_at[d]
    // vertices); the leaves of a node at level M-2 are its edges plus one listed edge each
    int len[5], nxt[5], nv_at[5];
    len[0] = over ? 0 : n0;
    nxt[0] = 0;
    nv_at[0] = 2;
    int d = 0;
    int64_t ops = 0;
    while (d >= 0 && !over) {
      if ((++ops & 255) == 0 && warp_past(cx.deadline)) {
        if (lane == 0) atomicOr(cx.err, 4);
        break;
      }
      if (d == cx.M - 2 || nxt[d] >= len[d]) {
        if (d == cx.M - 2) {  // the leaves, one per lane
          for (int i = lane; i < len[d]; i += 32)
            esu_leaf(cx, vs, nvs, sa, sb, ns, ext[d * EXTCAP + i]);
          if (lane == 0) {
            my_nodes += (unsigned long long)len[d];
            my_leaves += (unsigned long long)len[d];
          }
        }
        // back to the parent: its edges and vertices
        --d;
        if (d >= 0) {
          ns = d + 1;
          nvs = nv_at[d];
        }
        continue;
      }
      // the child through the next listed edge w
      const int i = nxt[d]++;
      const int32_t w = ext[d * EXTCAP + i];
      const int32_t a = cx.eu[w], b = cx.ev[w];
      int ia = -1, ib = -1;
      for (int q = 0; q < nvs; ++q) {
        if (vs[q] == a) ia = q;
        if (vs[q] == b) ib = q;
      }
      int32_t xnew = -1;
      if (ia < 0) {
        ia = nvs;
        xnew = a;
      } else if (ib < 0) {
        ib = nvs;
        xnew = b;
      }
      // the child's list: the tail after w, then the edges after e0 from the new endpoint to
      // vertices outside the node
      const int tail = len[d] - i - 1;
      for (int q = lane; q < tail; q += 32) ext[(d + 1) * EXTCAP + q] = ext[d * EXTCAP + i + 1 + q];
      int n1 = tail;
      if (xnew >= 0) {
        for (int64_t b0 = g.off[xnew]; b0 < g.off[xnew + 1]; b0 += 32) {
          const int64_t t = b0 + lane;
          bool keep = false;
          int64_t id = -1;
          if (t < g.off[xnew + 1]) {
            const int32_t y = __ldg(g.adj + t);
            id = __ldg(cx.eid + t);
            keep = id > e0;
            for (int q = 0; q < nvs && keep; ++q) keep = vs[q] != y;
          }
          const unsigned bal = __ballot_sync(FULL, keep);
          const int at = n1 + __popc(bal & ((1u << lane) - 1));
          if (keep && at < EXTCAP) ext[(d + 1) * EXTCAP + at] = (int32_t)id;
          n1 += __popc(bal);
        }
      }
      __syncwarp();
      if (n1 > EXTCAP) {
        over = true;
        break;
      }
      if (lane == 0) ++my_nodes;
      sa[ns] = (int8_t)ia;
      sb[ns] = (int8_t)ib;
      ++ns;
      if (xnew >= 0) vs[nvs++] = xnew;
      ++d;
      len[d] = n1;
      nxt[d] = 0;
      nv_at[d] = nvs;
    }
    if (over && lane == 0) atomicOr(cx.err, 1);
  }
  if (lane == 0) {
    atomicAdd(cx.nodes, my_nodes);
    atomicAdd(cx.leaves, my_leaves);
  }
}

__global__ void k_dom_popc(const uint32_t* __restrict__ dom, int64_t npat, int64_t words,
                           const unsigned long long* __restrict__ pat,
                           unsigned long long* __restrict__ mni) {
  // one warp per (pattern, position); positions past the pattern's size are skipped
  const int lane = threadIdx.x & 31;
  for (int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; w < npat * EPV;
       w += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    const int64_t p = w / EPV;
    const int pos = (int)(w % EPV);
    const int nv = (int)(pat[p] >> 61);
    if (pos >= nv) continue;
    const uint32_t* D = dom + (p * EPV + pos) * words;
    unsigned long long c = 0;
    for (int64_t i = lane; i < words; i += 32) c += __popc(D[i]);
    for (int o = 16; o; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if (lane == 0) atomicMin(mni + p, c);
  }
}

// flag[i] = 1 for an occupied slot of the hash set
__global__ void k_slot_flag(const unsigned long long* __restrict__ tab, int64_t n,
                            int64_t* __restrict__ flag) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    flag[i] = tab[i] != ~0ull ? 1 : 0;
}

__global__ void k_slot_scatter(const unsigned long long* __restrict__ tab, int64_t n,
                               const int64_t* __restrict__ flag, const int64_t* __restrict__ pos,
                               unsigned long long* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    if (flag[i]) out[pos[i]] = tab[i];
}

__global__ void k_iota64(int64_t* p, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    p[i] = i;
}

// sort key of pattern perm[i]: which = 0 its code, 1 the inverted support
__global__ void k_pat_key(const unsigned long long* __restrict__ pat,
                          const unsigned long long* __restrict__ mni,
                          const int64_t* __restrict__ perm, int64_t n, int which,
                          unsigned long long* __restrict__ key) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = perm[i];
    key[i] = which == 0 ? pat[p] : ~mni[p];
  }
}

__global__ void k_pat_gather(const unsigned long long* __restrict__ pat,
                             const unsigned long long* __restrict__ mni,
                             const int64_t* __restrict__ perm, int64_t n,
                             unsigned long long* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = perm[i];
    out[2 * i] = mni[p];
    out[2 * i + 1] = pat[p];
  }
}

inline int egrid(int64_t n) {
  return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, (int64_t)sm_count() * 32));
}

}  // namespace

void topk_patterns_edge(nuri_graph* G, int32_t M, int32_t k, uint32_t flags, cudaStream_t s,
                        nuri_result** out) {
  const DevGraph& g = G->d;
  DevTimer timer(s);
  const bool keep_ties = flags & NURI_KEEP_TIES;
  int64_t launches = 0;
  nuri_stats stats;
  memset(&stats, 0, sizeof(stats));
  const int64_t nnz = g.nnz;
  const int64_t words = ((int64_t)g.n + 31) / 32;

  // the edge list and the edge number of every CSR entry
  DBuf<int64_t> keep, pos, eid;
  keep.alloc(nnz + 1, s);
  pos.alloc(nnz + 1, s);
  eid.alloc(std::max<int64_t>(nnz, 1), s);
  NURI_CUDA(cudaMemsetAsync(keep.p, 0, sizeof(int64_t) * (nnz + 1), s));
  if (nnz > 0) {
    ++launches;
    k_edge_flags<<<egrid((int64_t)g.n * 32), 256, 0, s>>>(g, keep.p);
  }
  size_t tb = 0;
  cub::DeviceScan::ExclusiveSum(nullptr, tb, keep.p, pos.p, nnz + 1, s);
  DBuf<uint8_t> tmp;
  tmp.alloc(tb, s);
  NURI_CUDA(cub::DeviceScan::ExclusiveSum(tmp.p, tb, keep.p, pos.p, nnz + 1, s));
  int64_t m = 0;
  NURI_CUDA(cudaMemcpyAsync(&m, pos.p + nnz, 8, cudaMemcpyDeviceToHost, s));
  NURI_CUDA(cudaStreamSynchronize(s));
  DBuf<int32_t> eu, ev;
  eu.alloc(std::max<int64_t>(m, 1), s);
  ev.alloc(std::max<int64_t>(m, 1), s);
  if (nnz > 0) {
    ++launches;
    k_edge_ids<<<egrid((int64_t)g.n * 32), 256, 0, s>>>(g, pos.p, eu.p, ev.p, eid.p);
  }

  // bits per label in a packed code (up to 128 labels fit 64 bits with 6 vertices)
  int lb = 1;
  while ((1 << lb) < std::max(g.L, 2)) ++lb;
  if (lb > 7)
    NURI_FAIL(NURI_ERR_LIMIT, "nuri_topk_patterns: edge-oriented expansion takes at most 128 labels");
  const int grid = sm_count() * 2;
  const int64_t nwarps = (int64_t)grid * ESU_WARPS;
  constexpr int64_t kTable = 1 << 20;  // hash-set slots (patterns up to half of it)
  DBuf<int32_t> scratch, err;
  scratch.alloc(nwarps * M * EXTCAP, s);
  err.alloc(1, s);
  DBuf<unsigned long long> work, nodes, leaves, table;
  work.alloc(1, s);
  nodes.alloc(1, s);
  leaves.alloc(1, s);
  table.alloc(kTable, s);
  NURI_CUDA(cudaMemsetAsync(table.p, 0xff, 8 * kTable, s));
  DBuf<uint64_t> deadline;
  deadline.alloc(1, s);
  ++launches;
  k_set_deadline<<<1, 32, 0, s>>>(deadline.p, time_budget_ns());
  EsuCtx cx;
  memset(&cx, 0, sizeof(cx));
  cx.g = g;
  cx.eu = eu.p;
  cx.ev = ev.p;
  cx.eid = eid.p;
  cx.m = m;
  cx.M = M;
  cx.scratch = scratch.p;
  cx.work = work.p;
  cx.nodes = nodes.p;
  cx.leaves = leaves.p;
  cx.err = err.p;
  cx.deadline = deadline.p;
  cx.words = words;
  cx.table = table.p;
  cx.table_mask = kTable - 1;
  cx.lb = lb;
  NURI_CUDA(cudaMemsetAsync(err.p, 0, 4, s));

  auto run = [&](int pass) {
    cx.pass = pass;
    NURI_CUDA(cudaMemsetAsync(work.p, 0, 8, s));
    NURI_CUDA(cudaMemsetAsync(nodes.p, 0, 8, s));
    NURI_CUDA(cudaMemsetAsync(leaves.p, 0, 8, s));
    ++launches;
    ++stats.expand_launches;
    k_esu<<<grid, ESU_WARPS * 32, 0, s>>>(cx);
    NURI_CUDA(cudaGetLastError());
    int32_t e = 0;
    unsigned long long nn = 0, nl = 0;
    NURI_CUDA(cudaMemcpyAsync(&e, err.p, 4, cudaMemcpyDeviceToHost, s));
    NURI_CUDA(cudaMemcpyAsync(&nn, nodes.p, 8, cudaMemcpyDeviceToHost, s));
    NURI_CUDA(cudaMemcpyAsync(&nl, leaves.p, 8, cudaMemcpyDeviceToHost, s));
    NURI_CUDA(cudaStreamSynchronize(s));
    if (e & 4) NURI_FAIL(NURI_ERR_TIMEOUT, "nuri_topk_patterns: time budget exhausted");
    if (e & 1)
      NURI_FAIL(NURI_ERR_LIMIT,
                "nuri_topk_patterns: edge-oriented expansion: more than %d edges adjacent to a "
                "subgraph (degrees too high for this mode)", EXTCAP);
    if (e & 8)
      NURI_FAIL(NURI_ERR_LIMIT, "nuri_topk_patterns: edge-oriented expansion: too many patterns");
    if (pass == 1) {
      stats.expansions = (int64_t)nn;
      stats.results_stored = (int64_t)nl;  // embeddings
    }
  };

  // pass 1: the patterns (hash set of codes), compacted and sorted
  run(1);
  int64_t npat = 0;
  DBuf<unsigned long long> pat;
  {
    DBuf<int64_t> flag, fpos;
    flag.alloc(kTable + 1, s);
    fpos.alloc(kTable + 1, s);
    NURI_CUDA(cudaMemsetAsync(flag.p + kTable, 0, 8, s));
    ++launches;
    k_slot_flag<<<egrid(kTable), 256, 0, s>>>(table.p, kTable, flag.p);
    size_t t3 = 0;
    cub::DeviceScan::ExclusiveSum(nullptr, t3, flag.p, fpos.p, kTable + 1, s);
    DBuf<uint8_t> tmp3;
    tmp3.alloc(t3, s);
    NURI_CUDA(cub::DeviceScan::ExclusiveSum(tmp3.p, t3, flag.p, fpos.p, kTable + 1, s));
    NURI_CUDA(cudaMemcpyAsync(&npat, fpos.p + kTable, 8, cudaMemcpyDeviceToHost, s));
    NURI_CUDA(cudaStreamSynchronize(s));
    DBuf<unsigned long long> un;
    un.alloc(std::max<int64_t>(npat, 1), s);
    pat.alloc(std::max<int64_t>(npat, 1), s);
    ++launches;
    k_slot_scatter<<<egrid(kTable), 256, 0, s>>>(table.p, kTable, flag.p, fpos.p, un.p);
    if (npat > 0) {
      size_t t1 = 0;
      cub::DeviceRadixSort::SortKeys(nullptr, t1, un.p, pat.p, npat, 0, 64, s);
      DBuf<uint8_t> tmp1;
      tmp1.alloc(t1, s);
      NURI_CUDA(cub::DeviceRadixSort::SortKeys(tmp1.p, t1, un.p, pat.p, npat, 0, 64, s));
    }
  }
  table.reset();
  // pass 2: domains
  DBuf<uint32_t> dom;
  DBuf<unsigned long long> mni;
  if (npat > 0) {
    dom.alloc(npat * EPV * words, s);
    NURI_CUDA(cudaMemsetAsync(dom.p, 0, sizeof(uint32_t) * npat * EPV * words, s));
    cx.pat = pat.p;
    cx.npat = npat;
    cx.dom = dom.p;
    run(2);
    mni.alloc(npat, s);
    NURI_CUDA(cudaMemsetAsync(mni.p, 0xff, 8 * npat, s));
    ++launches;
    k_dom_popc<<<egrid(npat * EPV * 32), 256, 0, s>>>(dom.p, npat, words, pat.p, mni.p);
  }
  // rank: (support desc, code asc) by two stable radix passes
  std::vector<unsigned long long> ranked(2 * std::max<int64_t>(npat, 1));
  if (npat > 0) {
    DBuf<int64_t> perm, perm2;
    DBuf<unsigned long long> key, key2, outp;
    perm.alloc(npat, s);
    perm2.alloc(npat, s);
    key.alloc(npat, s);
    key2.alloc(npat, s);
    outp.alloc(2 * npat, s);
    ++launches;
    k_iota64<<<egrid(npat), 256, 0, s>>>(perm.p, npat);
    size_t t2 = 0;
    cub::DeviceRadixSort::SortPairs(nullptr, t2, key.p, key2.p, perm.p, perm2.p, npat, 0, 64, s);
    DBuf<uint8_t> tmp2;
    tmp2.alloc(t2, s);
    for (int which = 0; which < 2; ++which) {
      ++launches;
      k_pat_key<<<egrid(npat), 256, 0, s>>>(pat.p, mni.p, perm.p, npat, which, key.p);
      NURI_CUDA(cub::DeviceRadixSort::SortPairs(tmp2.p, t2, key.p, key2.p, perm.p, perm2.p, npat,
                                                0, 64, s));
      std::swap(perm.p, perm2.p);
    }
    ++launches;
    k_pat_gather<<<egrid(npat), 256, 0, s>>>(pat.p, mni.p, perm.p, npat, outp.p);
    NURI_CUDA(cudaMemcpyAsync(ranked.data(), outp.p, 8 * 2 * npat, cudaMemcpyDeviceToHost, s));
    NURI_CUDA(cudaStreamSynchronize(s));
  }
  int64_t count = std::min<int64_t>(npat, k);
  if (keep_ties && npat > k)
    while (count < npat && ranked[2 * count] == ranked[2 * (k - 1)]) ++count;
  // rows: labels and edges decoded from the packed codes
  const unsigned long long lmask = (1ull << lb) - 1;
  int64_t nverts = 0, nedges = 0;
  for (int64_t i = 0; i < count; ++i) {
    const unsigned long long key = ranked[2 * i + 1];
    nverts += (int)(key >> 61);
    nedges += __builtin_popcountll(key & 0x7fffull);
  }
  nuri_result* r = new_result(2, (int32_t)count, nverts, nedges, true);
  int64_t pv = 0, pe = 0;
  for (int64_t i = 0; i < count; ++i) {
    const unsigned long long key = ranked[2 * i + 1];
    const int nv = (int)(key >> 61);
    r->score[i] = (int64_t)ranked[2 * i];
    r->vert_off[i] = (int32_t)pv;
    r->edge_off[i] = (int32_t)pe;
    for (int x = 0; x < nv; ++x) {
      r->verts[pv] = x;
      r->labels[pv] = (int32_t)((key >> (61 - lb * (x + 1))) & lmask);
      ++pv;
    }
    const int ntri = nv * (nv - 1) / 2;
    int idx = 0;
    for (int a = 0; a < nv; ++a)
      for (int b = a + 1; b < nv; ++b, ++idx)
        if ((key >> (ntri - 1 - idx)) & 1) {
          r->edges[2 * pe] = a;
          r->edges[2 * pe + 1] = b;
          ++pe;
        }
  }
  r->vert_off[count] = (int32_t)pv;
  r->edge_off[count] = (int32_t)pe;
  stats.threshold = count > 0 ? (int64_t)ranked[2 * (count - 1)] : INT64_MIN;
  stats.dequeued = npat;
  stats.device_ms = timer.stop();
  stats.launches = launches;
  r->stats = stats;
  *out = r;
}

}  // namespace nuri
