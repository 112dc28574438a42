// Top-k cliques ranked by cumulative vertex weight.  Section 2's top-k semantics leaves the
// ranking criterion to the user; this is the clique search of Algorithm 1 (the clique
// functions of Section 3.2) with a weight sum as the score:
//
//   score(s)   = w(V_s), the sum of the int32 vertex weights (>= 0) of the clique
//   u(s)       = w(P_s): every clique below s adds a subset of its candidates P_s
//   dominated  = w(V_s) + w(P_s) < tau (strict), tau = a lower bound of the k-th best score
//   results    = every clique (or every maximal one); ties at the k-th place by sorted ids
//
// GPU organisation (ranks of the degeneracy orientation, as in the search by size):
//   * seeds: one per vertex r with P = N+(r) and bound w(r) + w(N+(r)), sorted by bound;
//   * k_wclique_expand: one warp per item (a seed or a record), taken in bound order.  P comes
//     from intersecting the members' out-rows.  |P| <= 64: the whole subtree is searched in
//     the warp on a 64 x 64 adjacency bitmap, the lanes taking the record's children one at a
//     time, each a depth-first search that drops a node when w(C) + w(candidates) < tau.
//     |P| > 64: one child per candidate d (the candidates after d adjacent to it, counted and
//     weighed with a ballot), kept when its bound reaches tau; a record whose children do not
//     fit the launch's output is handed back whole;
//   * host: a stack of sorted batches (depth first, highest bounds on top), so the records in
//     flight stay few;
//   * tau: the k-th largest vertex weight to start with (every vertex is a clique), then from
//     a histogram of score >> shift, raised with atomicMax;
//   * top-k merge: rows with score >= tau; least-significant-column-first radix passes over
//     the sorted ids, then over the score (descending).
#include <cub/cub.cuh>

#include <algorithm>
#include <climits>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "nuri_internal.cuh"
#include "topk_common.cuh"

namespace nuri {
namespace {

constexpr int WMAXD = 256;        // largest clique a row holds (NURI_ERR_LIMIT above)
constexpr int WBINS = 16384;      // threshold histogram bins (score >> shift)
constexpr int WWARPS = 4;         // warps per block of the expansion kernel
constexpr int WSEG = 512;         // candidates a warp keeps in shared memory
constexpr int64_t kBatch = 1 << 16;     // items per launch
constexpr int64_t kOutCap = 1 << 18;    // child records per launch

struct WRec {
  long long key;  // frontier: bound; result: score
  int32_t nv;
  int32_t pad;
  int32_t V[WMAXD];  // ranks
};

struct WState {
  long long tau;
  unsigned long long res_count, out_count, defer_count, work_next;
  unsigned long long expansions, pruned, dequeued, adj_bytes;
  int32_t hmax, err;  // err bit 0: a clique above WMAXD; bit 2: time budget exhausted;
                      // bit 3: a frontier record that is not one (internal error)
};

struct WCtx {
  DevGraph g;
  const int32_t* wr;  // weight of every rank
  WState* st;
  int32_t* hist;      // WBINS
  WRec* res;
  int64_t res_cap;
  WRec* out;          // children of this launch
  int64_t out_cap;
  WRec* defer;        // items handed back whole
  int32_t* scratch;   // per warp: max_out candidates (rows longer than WSEG)
  int64_t k;
  int32_t shift, maximal, no_prune;
  const uint64_t* deadline;
};

__device__ __forceinline__ long long ld_volatile64(const long long* p) {
  return *(const volatile long long*)p;
}

__device__ __forceinline__ int64_t lower_bound64(const int32_t* a, int64_t lo, int64_t hi,
                                                 int32_t x) {
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (__ldg(a + mid) < x) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

__device__ __forceinline__ bool has_out(const DevGraph& g, int32_t a, int32_t b) {
  // b in the out-row of a (ranks above a, sorted)
  const int64_t e = g.ooff[a + 1];
  const int64_t p = lower_bound64(g.oout, g.ooff[a], e, b);
  return p < e && __ldg(g.oout + p) == b;
}

// Is the clique C (ranks) maximal in the whole graph?  No vertex adjacent to every member:
// the undirected row (original ids) of the member with the fewest neighbours is scanned.
__device__ bool w_is_maximal(const DevGraph& g, const int32_t* C, int nv) {
  int best = 0;
  int64_t blen = INT64_MAX;
  for (int i = 0; i < nv; ++i) {
    const int32_t v = g.vert_of[C[i]];
    const int64_t len = g.off[v + 1] - g.off[v];
    if (len < blen) {
      blen = len;
      best = i;
    }
  }
  const int32_t v0 = g.vert_of[C[best]];
  for (int64_t t = g.off[v0]; t < g.off[v0 + 1]; ++t) {
    const int32_t x = g.adj[t];
    bool all = true;
    for (int i = 0; i < nv && all; ++i) {
      if (i == best) continue;
      const int32_t u = g.vert_of[C[i]];
      if (u == x) {
        all = false;
        break;
      }
      const int64_t e = g.off[u + 1];
      const int64_t p = lower_bound64(g.adj, g.off[u], e, x);
      all = p < e && __ldg(g.adj + p) == x;
    }
    if (all) return false;
  }
  return true;
}

// Append a result (the record's members V[0..nv) and extra[0..ne)) and refresh tau.  Any
// snapshot of the histogram undercounts the final one, so the published value (the lower edge
// of the bin where the count from the top reaches k) never exceeds the k-th best score.
__device__ void w_add_result(const WCtx& cx, const int32_t* V, int nv, const int32_t* extra,
                             int ne, long long score) {
  WState* S = cx.st;
  const unsigned long long slot = atomicAdd(&S->res_count, 1ull);
  if ((int64_t)slot < cx.res_cap) {
    WRec* r = cx.res + slot;
    r->key = score;
    r->nv = nv + ne;
    for (int i = 0; i < nv; ++i) r->V[i] = V[i];
    for (int i = 0; i < ne; ++i) r->V[nv + i] = extra[i];
  }
  const long long bl = score >> cx.shift;
  const int32_t bin = bl >= WBINS ? WBINS - 1 : (int32_t)bl;
  atomicAdd(cx.hist + bin, 1);
  if (bin > *(volatile int32_t*)&S->hmax) atomicMax(&S->hmax, bin);
  if ((int64_t)slot + 1 < cx.k || (slot & 7) != 0) return;  // every 8th result refreshes
  const long long cur = ld_volatile64(&S->tau);
  const int32_t floor_bin = cur <= 0 ? 0 : (int32_t)min(cur >> cx.shift, (long long)WBINS - 1);
  long long acc = 0;
  for (int32_t b = *(volatile int32_t*)&S->hmax; b >= floor_bin; --b) {
    acc += *(volatile int32_t*)(cx.hist + b);
    if (acc >= cx.k) {
      const long long t = (long long)b << cx.shift;
      if (t > cur) atomicMax(&S->tau, t);
      return;
    }
  }
}

__global__ void k_wrank_weights(const int32_t* __restrict__ vert_of,
                                const int32_t* __restrict__ weights, int32_t n,
                                int32_t* __restrict__ wr) {
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n;
       r += (int64_t)gridDim.x * blockDim.x)
    wr[r] = weights[vert_of[r]];
}

// one warp per rank: bound = w(r) + w(N+(r))
__global__ void k_wseed_bounds(DevGraph g, const int32_t* __restrict__ wr,
                               long long* __restrict__ keys, int32_t* __restrict__ vals) {
  const int lane = threadIdx.x & 31;
  for (int64_t r = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; r < g.n;
       r += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    long long s = 0;
    for (int64_t t = g.ooff[r] + lane; t < g.ooff[r + 1]; t += 32) s += __ldg(wr + g.oout[t]);
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) {
      keys[r] = s + wr[r];
      vals[r] = (int32_t)r;
    }
  }
}

__global__ void __launch_bounds__(WWARPS * 32) k_wclique_expand(WCtx cx,
                                                                const WRec* __restrict__ in,
                                                                const int32_t* __restrict__ seeds,
                                                                const long long* __restrict__ seed_keys,
                                                                int64_t nin) {
  __shared__ int32_t sV[WWARPS][WMAXD];
  __shared__ int32_t sP[WWARPS][WSEG];
  __shared__ unsigned long long sRow[WWARPS][64];
  __shared__ int32_t sW[WWARPS][64];
  __shared__ int32_t sNext[WWARPS];
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const DevGraph& g = cx.g;
  const int64_t gwarp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  int32_t* scratch = cx.scratch + gwarp * (int64_t)max(g.max_out, 1);
  unsigned long long my_exp = 0, my_pruned = 0, my_deq = 0, my_bytes = 0;
  bool limit = false;
  while (true) {
    long long item = 0;
    __syncwarp();
    if (lane == 0) {
      item = (long long)atomicAdd(&cx.st->work_next, 1ull);
      if (item < nin && global_ns() > *(const volatile uint64_t*)cx.deadline) {
        atomicOr(&cx.st->err, 4);
        item = nin;
      }
    }
    item = __shfl_sync(FULL, item, 0);
    if (item >= nin) break;
    int nv;
    long long key;
    if (seeds) {
      nv = 1;
      key = seed_keys[item];
      if (lane == 0) sV[w][0] = seeds[item];
    } else {
      nv = in[item].nv;
      key = in[item].key;
      if (nv < 1 || nv > WMAXD) {  // not a record (cannot happen): reported, never followed
        if (lane == 0) atomicOr(&cx.st->err, 8);
        continue;
      }
      for (int i = lane; i < nv; i += 32) sV[w][i] = in[item].V[i];
    }
    __syncwarp();
    const long long tau = warp_load(&cx.st->tau);  // one value for the warp's branches
    if (nv <= 0 || (!cx.no_prune && key < tau)) {  // an empty slot, or dominated
      if (lane == 0 && nv > 0) ++my_pruned;
      continue;
    }
    if (lane == 0) ++my_deq;
    // ---- candidates P: ranks after the last member, adjacent to every member ----
    const int32_t last = sV[w][nv - 1];
    int64_t cb = g.ooff[last], ce = g.ooff[last + 1];
    int srci = nv - 1;
    for (int i = 0; i < nv - 1; ++i) {
      const int32_t v = sV[w][i];
      const int64_t re = g.ooff[v + 1];
      const int64_t rb = lower_bound64(g.oout, g.ooff[v], re, last + 1);
      if (re - rb < ce - cb) {
        cb = rb;
        ce = re;
        srci = i;
      }
    }
    int32_t* P = (ce - cb) <= WSEG ? sP[w] : scratch;
    int p = 0;
    for (int64_t base = cb; base < ce; base += 32) {
      const int64_t t = base + lane;
      bool keep = false;
      int32_t x = 0;
      if (t < ce) {
        x = __ldg(g.oout + t);
        keep = x > last;
        for (int i = 0; i < nv && keep; ++i)
          if (i != srci) keep = has_out(g, sV[w][i], x);
      }
      const unsigned bal = __ballot_sync(FULL, keep);
      if (keep) P[p + __popc(bal & ((1u << lane) - 1))] = x;
      p += __popc(bal);
    }
    __syncwarp();
    if (lane == 0) my_bytes += 4ull * (unsigned long long)(ce - cb) * nv;
    long long wv = 0;
    for (int i = lane; i < nv; i += 32) wv += __ldg(cx.wr + sV[w][i]);
    for (int o = 16; o; o >>= 1) wv += __shfl_xor_sync(FULL, wv, o);
    if (nv >= WMAXD && p > 0) {
      if (lane == 0) atomicOr(&cx.st->err, 1);
      continue;
    }
    // ---- a record with many candidates: its children go to the output, all or none ----
    int64_t base_slot = 0;
    if (p > 64) {
      int ok = 1;
      if (lane == 0) {
        base_slot = (int64_t)atomicAdd(&cx.st->out_count, (unsigned long long)p);
        if (base_slot + p > cx.out_cap) {
          ok = 0;
          const int64_t ds = (int64_t)atomicAdd(&cx.st->defer_count, 1ull);
          WRec* r = cx.defer + ds;
          r->key = key;
          r->nv = nv;
          for (int i = 0; i < nv; ++i) r->V[i] = sV[w][i];
          --my_deq;
        }
      }
      ok = __shfl_sync(FULL, ok, 0);
      base_slot = __shfl_sync(FULL, base_slot, 0);
      if (!ok) continue;
    }
    // ---- the record itself is a result ----
    if (lane == 0 && wv >= tau && (!cx.maximal || (p == 0 && w_is_maximal(g, sV[w], nv))))
      w_add_result(cx, sV[w], nv, nullptr, 0, wv);
    if (p == 0) continue;
    if (p > 64) {
      for (int j = 0; j < p; ++j) {
        const int32_t d = P[j];
        // the weight of the candidates after d adjacent to d
        long long ws = 0;
        for (int t = j + 1 + lane; t < p; t += 32)
          if (has_out(g, d, P[t])) ws += __ldg(cx.wr + P[t]);
        for (int o = 16; o; o >>= 1) ws += __shfl_xor_sync(FULL, ws, o);
        if (lane == 0) {
          ++my_exp;
          my_bytes += 4ull * (unsigned long long)(p - j);
          WRec* r = cx.out + base_slot + j;
          const long long bound = wv + __ldg(cx.wr + d) + ws;
          if (!cx.no_prune && bound < ld_volatile64(&cx.st->tau)) {
            ++my_pruned;
            r->nv = 0;
          } else {
            r->key = bound;
            r->nv = nv + 1;
            for (int i = 0; i < nv; ++i) r->V[i] = sV[w][i];
            r->V[nv] = d;
          }
        }
      }
      __syncwarp();
      continue;
    }
    // ---- at most 64 candidates: the subtree in this warp on bitmap rows ----
    if (P != sP[w]) {
      for (int i = lane; i < p; i += 32) sP[w][i] = P[i];
      __syncwarp();
    }
    const int32_t* sp = sP[w];
    const int32_t plast = sp[p - 1];
    for (int i = lane; i < p; i += 32) {
      sRow[w][i] = 0ull;
      sW[w][i] = __ldg(cx.wr + sp[i]);
    }
    __syncwarp();
    // row i: the candidates j > i in the out-row of candidate i
    for (int i = 0; i < p; ++i) {
      const int64_t rb = g.ooff[sp[i]], re = g.ooff[sp[i] + 1];
      for (int64_t b0 = rb; b0 < re; b0 += 32) {
        const int64_t t = b0 + lane;
        const int32_t x = t < re ? __ldg(g.oout + t) : INT32_MAX;
        if (x <= plast) {
          int lo = i + 1, hi = p;
          while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (sp[mid] < x) lo = mid + 1;
            else hi = mid;
          }
          if (lo < p && sp[lo] == x) atomicOr(&sRow[w][i], 1ull << lo);
        }
        if (__all_sync(FULL, x > plast)) break;
      }
    }
    if (lane == 0) {
      my_bytes += 4ull * (unsigned long long)p * 2;
      sNext[w] = 0;
    }
    __syncwarp();
    // lanes take the record's children dynamically; each searches its child's subtree
    int32_t ext[65];
    unsigned long long K[65], T[65];
    long long WC[65];
    bool stop = false;
    while (!stop) {
      const int i = atomicAdd(&sNext[w], 1);
      if (i >= p) break;
      int d = 0;
      ext[0] = sp[i];
      K[0] = sRow[w][i];
      WC[0] = wv + sW[w][i];
      bool visit = true;
      while (d >= 0) {
        if (visit) {
          visit = false;
          ++my_exp;
          if ((my_exp & 1023) == 0 && global_ns() > *(const volatile uint64_t*)cx.deadline) {
            atomicOr(&cx.st->err, 4);
            stop = true;
            break;
          }
          const long long tnow = ld_volatile64(&cx.st->tau);
          if (nv + d + 1 > WMAXD) {
            limit = true;
            T[d] = 0;
          } else {
            if (WC[d] >= tnow) {
              bool rel = true;
              if (cx.maximal) {
                rel = false;
                if (K[d] == 0ull) {
                  int32_t C[WMAXD];
                  for (int a = 0; a < nv; ++a) C[a] = sV[w][a];
                  for (int a = 0; a <= d; ++a) C[nv + a] = ext[a];
                  rel = w_is_maximal(g, C, nv + d + 1);
                }
              }
              if (rel) w_add_result(cx, sV[w], nv, ext, d + 1, WC[d]);
            }
            long long bound = WC[d];
            for (unsigned long long m = K[d]; m; m &= m - 1) bound += sW[w][__ffsll((long long)m) - 1];
            if (!cx.no_prune && bound < ld_volatile64(&cx.st->tau)) {
              if (K[d]) ++my_pruned;
              T[d] = 0;
            } else {
              T[d] = K[d];
            }
          }
        }
        if (T[d] == 0ull) {
          --d;
          continue;
        }
        const int j = __ffsll((long long)T[d]) - 1;
        T[d] &= T[d] - 1;
        if (d + 1 >= 64) {  // cannot happen: at most 64 candidates
          limit = true;
          continue;
        }
        ext[d + 1] = sp[j];
        K[d + 1] = K[d] & sRow[w][j];
        WC[d + 1] = WC[d] + sW[w][j];
        ++d;
        visit = true;
      }
    }
    __syncwarp();
  }
  if (limit) atomicOr(&cx.st->err, 1);
  for (int o = 16; o; o >>= 1) {
    my_exp += __shfl_xor_sync(FULL, my_exp, o);
    my_pruned += __shfl_xor_sync(FULL, my_pruned, o);
  }
  if (lane == 0) {
    atomicAdd(&cx.st->expansions, my_exp);
    atomicAdd(&cx.st->pruned, my_pruned);
    atomicAdd(&cx.st->dequeued, my_deq);
    atomicAdd(&cx.st->adj_bytes, my_bytes);
  }
}

// rows with key >= tau (and nv > 0) compacted into out
__global__ void k_wcompact(const WRec* __restrict__ in, int64_t n, long long tau,
                           WRec* __restrict__ out, unsigned long long* cnt) {
  const int lane = threadIdx.x & 31;
  for (int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; i < n;
       i += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    const int nv = in[i].nv;
    if (nv <= 0 || in[i].key < tau) continue;
    unsigned long long slot = 0;
    if (lane == 0) slot = atomicAdd(cnt, 1ull);
    slot = __shfl_sync(0xffffffffu, slot, 0);
    if (lane == 0) {
      out[slot].key = in[i].key;
      out[slot].nv = nv;
    }
    for (int a = lane; a < nv; a += 32) out[slot].V[a] = in[i].V[a];
  }
}

// Slots of the launch output marked empty: a record whose reservation fails still moves the
// output counter, so slots past the last granted reservation are read by the compaction and
// must not hold records of an earlier launch.
__global__ void k_wclear(WRec* __restrict__ recs, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    recs[i].nv = 0;
}

__global__ void k_wkeys(const WRec* __restrict__ recs, int64_t n, long long* __restrict__ keys,
                        int32_t* __restrict__ idx) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    keys[i] = recs[i].key;
    idx[i] = (int32_t)i;
  }
}

__global__ void k_wgather(const WRec* __restrict__ in, const int32_t* __restrict__ idx, int64_t n,
                          WRec* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  for (int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; i < n;
       i += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    const WRec& r = in[idx[i]];
    if (lane == 0) {
      out[i].key = r.key;
      out[i].nv = r.nv;
    }
    for (int a = lane; a < r.nv; a += 32) out[i].V[a] = r.V[a];
  }
}

// final selection: rows with score >= tau, their members as sorted original ids
__global__ void k_wselect(const WRec* __restrict__ res, int64_t cnt, long long tau,
                          const int32_t* __restrict__ vert_of, int32_t* __restrict__ selV,
                          int32_t* __restrict__ selN, long long* __restrict__ selS,
                          int32_t* nsel) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < cnt;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int c = res[i].nv;
    if (c <= 0 || c > WMAXD || res[i].key < tau) continue;
    const int pos = atomicAdd(nsel, 1);
    int32_t* ids = selV + (int64_t)pos * WMAXD;
    for (int t = 0; t < c; ++t) ids[t] = __ldg(vert_of + res[i].V[t]);
    for (int a = 1; a < c; ++a) {
      const int32_t x = ids[a];
      int b = a - 1;
      while (b >= 0 && ids[b] > x) {
        ids[b + 1] = ids[b];
        --b;
      }
      ids[b + 1] = x;
    }
    selN[pos] = c;
    selS[pos] = res[i].key;
  }
}

__global__ void k_wmax_rows(const int32_t* __restrict__ selN, int32_t n, int32_t* out) {
  int32_t best = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    best = max(best, selN[i]);
  for (int o = 16; o; o >>= 1) best = max(best, __shfl_xor_sync(0xffffffffu, best, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, best);
}

__global__ void k_wsorted_scores(const long long* __restrict__ selS,
                                 const int32_t* __restrict__ perm, int32_t n,
                                 long long* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = selS[perm[i]];
}

__global__ void k_wiota(int32_t* p, int32_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    p[i] = (int32_t)i;
}

// sort key of column col of row perm[i]: id + 1 (0 past the row's end: a prefix ranks
// first); col = -1: the score's low word, -2: its high word, both inverted (descending)
__global__ void k_wcol(const int32_t* __restrict__ selV, const int32_t* __restrict__ selN,
                       const long long* __restrict__ selS, const int32_t* __restrict__ perm,
                       int32_t n, int col, uint32_t* __restrict__ key) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t r = perm[i];
    uint32_t k;
    if (col == -1) k = ~(uint32_t)((unsigned long long)selS[r] & 0xffffffffull);
    else if (col == -2) k = ~(uint32_t)((unsigned long long)selS[r] >> 32);
    else k = col < selN[r] ? (uint32_t)selV[(int64_t)r * WMAXD + col] + 1u : 0u;
    key[i] = k;
  }
}

__global__ void k_wemit(const int32_t* __restrict__ selV, const int32_t* __restrict__ selN,
                        const long long* __restrict__ selS, const int32_t* __restrict__ perm,
                        int32_t count, const int32_t* __restrict__ off, int32_t* __restrict__ outV,
                        long long* __restrict__ outS) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t r = perm[i];
    for (int t = 0; t < selN[r]; ++t) outV[off[i] + t] = selV[(int64_t)r * WMAXD + t];
    outS[i] = selS[r];
  }
}

__global__ void k_wsizes(const int32_t* __restrict__ selN, const int32_t* __restrict__ perm,
                         int32_t count, int32_t* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = selN[perm[i]];
}

inline int wgrid(int64_t n) {
  return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, (int64_t)sm_count() * 32));
}

// A batch of items on the host's stack: seeds [s0, s1) of the sorted seed list, or records.
struct Batch {
  int64_t s0 = 0, s1 = 0;
  DBuf<WRec> recs;
  int64_t n = 0;
};

}  // namespace

int64_t wclique_query_bytes(const nuri_graph* G, int32_t k) {
  const int64_t n = std::max<int64_t>(G->d.n, 1);
  const int64_t warps = (int64_t)sm_count() * 8 * WWARPS;
  const int64_t res = std::max<int64_t>(1 << 16, (int64_t)k * 64);
  // seeds and their sort, rank weights, scratch, one launch's output and hand-back, the
  // result set (twice during a compaction) and the final merge; the stack of sorted batches
  // is not bounded in advance (deep searches hold more)
  return n * (8 * 2 + 4 * 2 + 4) + warps * (int64_t)std::max(G->d.max_out, 1) * 4 +
         (kOutCap + kBatch) * (int64_t)sizeof(WRec) * 2 +
         res * ((int64_t)sizeof(WRec) * 2 + 4 * WMAXD + 32) + (int64_t)WBINS * 4;
}

void topk_wcliques(nuri_graph* G, int32_t k, uint32_t flags, cudaStream_t s,
                   nuri_result** out) {
  const DevGraph& g = G->d;
  if (!g.weights) NURI_FAIL(NURI_ERR_INVALID, "nuri_topk_cliques: graph has no weights");
  DevTimer timer(s);
  int64_t launches = 0;
  const bool maximal = flags & NURI_CLIQUE_MAXIMAL;
  const bool no_prune = flags & NURI_NO_PRUNE;
  const bool keep_ties = flags & NURI_KEEP_TIES;
  const int32_t n = g.n;
  nuri_stats stats;
  memset(&stats, 0, sizeof(stats));

  DBuf<int32_t> wr, seeds, seeds2;
  DBuf<long long> skeys, skeys2;
  wr.alloc(std::max(n, 1), s);
  seeds.alloc(std::max(n, 1), s);
  seeds2.alloc(std::max(n, 1), s);
  skeys.alloc(std::max(n, 1), s);
  skeys2.alloc(std::max(n, 1), s);
  long long tau0 = LLONG_MIN;
  int64_t maxscore = 0;
  if (n > 0) {
    ++launches;
    k_wrank_weights<<<wgrid(n), 256, 0, s>>>(g.vert_of, g.weights, n, wr.p);
    ++launches;
    k_wseed_bounds<<<wgrid((int64_t)n * 32), 256, 0, s>>>(g, wr.p, skeys.p, seeds.p);
    size_t tb = 0;
    cub::DeviceRadixSort::SortPairsDescending(nullptr, tb, skeys.p, skeys2.p, seeds.p, seeds2.p,
                                              n, 0, 64, s);
    DBuf<uint8_t> tmp;
    tmp.alloc(tb, s);
    NURI_CUDA(cub::DeviceRadixSort::SortPairsDescending(tmp.p, tb, skeys.p, skeys2.p, seeds.p,
                                                        seeds2.p, n, 0, 64, s));
    // the k-th largest vertex weight (every vertex is a clique; all-cliques ranking only),
    // and the largest seed bound (no clique weighs more: it bounds the histogram's range)
    DBuf<int32_t> wsorted;
    wsorted.alloc(n, s);
    size_t tb2 = 0;
    cub::DeviceRadixSort::SortKeysDescending(nullptr, tb2, wr.p, wsorted.p, n, 0, 32, s);
    if (tb2 > tb) {
      tmp.alloc(tb2, s);
      tb = tb2;
    }
    NURI_CUDA(cub::DeviceRadixSort::SortKeysDescending(tmp.p, tb, wr.p, wsorted.p, n, 0, 32, s));
    int32_t kth = 0;
    long long top = 0;
    if (k <= n) NURI_CUDA(cudaMemcpyAsync(&kth, wsorted.p + (k - 1), 4, cudaMemcpyDeviceToHost, s));
    NURI_CUDA(cudaMemcpyAsync(&top, skeys2.p, 8, cudaMemcpyDeviceToHost, s));
    NURI_CUDA(cudaStreamSynchronize(s));
    if (k <= n && !maximal && !no_prune) tau0 = kth;
    maxscore = top;
  }
  int shift = 0;
  while ((maxscore >> shift) >= WBINS) ++shift;

  const int grid = sm_count() * 8;
  DBuf<WState> st;
  st.alloc(1, s);
  DBuf<int32_t> hist, scratch;
  hist.alloc(WBINS, s);
  scratch.alloc((int64_t)grid * WWARPS * std::max(g.max_out, 1), s);
  DBuf<uint64_t> deadline;
  deadline.alloc(1, s);
  ++launches;
  k_set_deadline<<<1, 32, 0, s>>>(deadline.p, time_budget_ns());
  // output slots per launch (a smaller value exercises the hand-back of records in tests)
  int64_t out_cap = kOutCap;
  if (const char* e = getenv("NURI_WOUT_CAP"))
    out_cap = std::max<int64_t>((int64_t)g.max_out + 1, std::min<int64_t>(kOutCap, atoll(e)));
  DBuf<WRec> outb, defer, res;
  outb.alloc(out_cap, s);
  defer.alloc(kBatch, s);
  int64_t res_cap = std::max<int64_t>(1 << 16, (int64_t)k * 64);
  if (const char* e = getenv("NURI_RESULT_CAP")) res_cap = std::max<int64_t>(1, atoll(e));
  DBuf<unsigned long long> cnt;
  cnt.alloc(1, s);
  DBuf<long long> bk1, bk2;
  DBuf<int32_t> bi1, bi2;
  DBuf<uint8_t> btmp;
  size_t btmp_bytes = 0;

  WCtx cx;
  memset(&cx, 0, sizeof(cx));
  cx.g = g;
  cx.wr = wr.p;
  cx.hist = hist.p;
  cx.out = outb.p;
  cx.out_cap = out_cap;
  cx.defer = defer.p;
  cx.scratch = scratch.p;
  cx.k = k;
  cx.shift = shift;
  cx.maximal = maximal;
  cx.no_prune = no_prune;
  cx.deadline = deadline.p;

  WState hs;
  int restarts = 0;
  while (true) {  // one pass; repeated only after a launch overflowed the result set
    res.alloc(res_cap, s);
    cx.res = res.p;
    cx.res_cap = res_cap;
    cx.st = st.p;
    memset(&hs, 0, sizeof(hs));
    hs.tau = tau0;
    NURI_CUDA(cudaMemcpyAsync(st.p, &hs, sizeof(hs), cudaMemcpyHostToDevice, s));
    NURI_CUDA(cudaMemsetAsync(hist.p, 0, sizeof(int32_t) * WBINS, s));
    ++launches;
    k_wclear<<<wgrid(out_cap), 256, 0, s>>>(outb.p, out_cap);  // no records of a past pass
    // the stack: seed batches, the best bounds on top
    std::vector<Batch> stack;
    for (int64_t b = ((int64_t)n + kBatch - 1) / kBatch - 1; b >= 0; --b) {
      Batch x;
      x.s0 = b * kBatch;
      x.s1 = std::min<int64_t>(n, x.s0 + kBatch);
      stack.push_back(std::move(x));
    }
    bool overflow = false;
    while (!stack.empty()) {
      Batch cur = std::move(stack.back());
      stack.pop_back();
      const bool is_seeds = cur.recs.p == nullptr;
      const int64_t nin = is_seeds ? cur.s1 - cur.s0 : cur.n;
      if (nin <= 0) continue;
      // out_count, defer_count, work_next (adjacent fields)
      NURI_CUDA(cudaMemsetAsync(&st.p->out_count, 0, 3 * sizeof(unsigned long long), s));
      ++launches;
      ++stats.expand_launches;
      k_wclique_expand<<<grid, WWARPS * 32, 0, s>>>(
          cx, cur.recs.p, is_seeds ? seeds2.p + cur.s0 : nullptr,
          is_seeds ? skeys2.p + cur.s0 : nullptr, nin);
      NURI_CUDA(cudaGetLastError());
      NURI_CUDA(cudaMemcpyAsync(&hs, st.p, sizeof(hs), cudaMemcpyDeviceToHost, s));
      NURI_CUDA(cudaStreamSynchronize(s));
      ++stats.rounds;
      if (hs.err & 8)
        NURI_FAIL(NURI_ERR_CUDA, "nuri_topk_cliques: internal error: a corrupt frontier record");
      if (hs.err & 1)
        NURI_FAIL(NURI_ERR_LIMIT, "nuri_topk_cliques: a clique exceeds %d vertices", WMAXD);
      if (hs.err & 4)
        NURI_FAIL(NURI_ERR_TIMEOUT, "nuri_topk_cliques: time budget exhausted (%llu nodes)",
                  (unsigned long long)hs.expansions);
      if ((int64_t)hs.res_count > res_cap) {
        overflow = true;
        break;
      }
      // results: compact once half full (rows below tau are never needed)
      if ((int64_t)hs.res_count > res_cap / 2) {
        NURI_CUDA(cudaMemsetAsync(cnt.p, 0, 8, s));
        DBuf<WRec> nb;
        nb.alloc(res_cap, s);
        ++launches;
        k_wcompact<<<wgrid((int64_t)hs.res_count * 32), 256, 0, s>>>(res.p, hs.res_count,
                                                                     hs.tau, nb.p, cnt.p);
        unsigned long long kept = 0;
        NURI_CUDA(cudaMemcpyAsync(&kept, cnt.p, 8, cudaMemcpyDeviceToHost, s));
        NURI_CUDA(cudaStreamSynchronize(s));
        if ((int64_t)kept * 2 > res_cap) {  // the rows at or above tau need more room
          const int64_t cap2 = (int64_t)kept * 4;
          DBuf<WRec> big;
          big.alloc(cap2, s);
          if (kept)
            NURI_CUDA(cudaMemcpyAsync(big.p, nb.p, sizeof(WRec) * kept, cudaMemcpyDeviceToDevice, s));
          nb = std::move(big);
          res_cap = cap2;
        }
        res = std::move(nb);
        cx.res = res.p;
        cx.res_cap = res_cap;
        const unsigned long long kept64 = kept;
        NURI_CUDA(cudaMemcpyAsync(&st.p->res_count, &kept64, 8, cudaMemcpyHostToDevice, s));
      }
      // records handed back go on the stack first (below the children: the children are the
      // deeper, more promising part), then the children sorted by bound
      if (hs.defer_count > 0) {
        Batch x;
        x.n = (int64_t)hs.defer_count;
        x.recs.alloc(x.n, s);
        NURI_CUDA(cudaMemcpyAsync(x.recs.p, defer.p, sizeof(WRec) * x.n, cudaMemcpyDeviceToDevice, s));
        stack.push_back(std::move(x));
      }
      const int64_t nout = std::min<int64_t>((int64_t)hs.out_count, out_cap);
      if (nout > 0) {
        // drop empty and dominated slots, then sort by bound descending
        DBuf<WRec> packed;
        packed.alloc(nout, s);
        NURI_CUDA(cudaMemsetAsync(cnt.p, 0, 8, s));
        ++launches;
        k_wcompact<<<wgrid(nout * 32), 256, 0, s>>>(outb.p, nout, no_prune ? LLONG_MIN : hs.tau,
                                                    packed.p, cnt.p);
        ++launches;
        k_wclear<<<wgrid(nout), 256, 0, s>>>(outb.p, nout);
        unsigned long long np = 0;
        NURI_CUDA(cudaMemcpyAsync(&np, cnt.p, 8, cudaMemcpyDeviceToHost, s));
        NURI_CUDA(cudaStreamSynchronize(s));
        if (np > 0) {
          if ((int64_t)bk1.n < (int64_t)np) {
            bk1.alloc(np, s);
            bk2.alloc(np, s);
            bi1.alloc(np, s);
            bi2.alloc(np, s);
          }
          ++launches;
          k_wkeys<<<wgrid(np), 256, 0, s>>>(packed.p, np, bk1.p, bi1.p);
          size_t tb = 0;
          cub::DeviceRadixSort::SortPairsDescending(nullptr, tb, bk1.p, bk2.p, bi1.p, bi2.p,
                                                    (int64_t)np, 0, 64, s);
          if (tb > btmp_bytes) {
            btmp.alloc(tb, s);
            btmp_bytes = tb;
          }
          NURI_CUDA(cub::DeviceRadixSort::SortPairsDescending(btmp.p, tb, bk1.p, bk2.p, bi1.p,
                                                              bi2.p, (int64_t)np, 0, 64, s));
          // batches of at most kBatch records, the lowest bounds pushed first
          for (int64_t b = ((int64_t)np + kBatch - 1) / kBatch - 1; b >= 0; --b) {
            Batch x;
            const int64_t b0 = b * kBatch, bn = std::min<int64_t>((int64_t)np - b0, kBatch);
            x.n = bn;
            x.recs.alloc(bn, s);
            ++launches;
            k_wgather<<<wgrid(bn * 32), 256, 0, s>>>(packed.p, bi2.p + b0, bn, x.recs.p);
            stack.push_back(std::move(x));
          }
        }
      }
      NURI_CUDA(cudaGetLastError());
    }
    if (overflow) {
      // every row at or above the final tau was counted: re-run from that tau with room
      tau0 = std::max(tau0, hs.tau);
      res_cap = std::max<int64_t>((int64_t)hs.res_count + 1024, res_cap * 2);
      ++restarts;
      NURI_CUDA(cudaStreamSynchronize(s));
      continue;
    }
    break;
  }

  // ---- top-k merge: rows with score >= tau, (score desc, sorted ids asc) ----
  NURI_CUDA(cudaMemcpyAsync(&hs, st.p, sizeof(hs), cudaMemcpyDeviceToHost, s));
  NURI_CUDA(cudaStreamSynchronize(s));
  const int64_t cntr = std::min<int64_t>((int64_t)hs.res_count, res_cap);
  const long long tau = hs.tau;
  DBuf<int32_t> selV, selN, nsel;
  DBuf<long long> selS;
  selV.alloc(std::max<int64_t>(cntr, 1) * WMAXD, s);
  selN.alloc(std::max<int64_t>(cntr, 1), s);
  selS.alloc(std::max<int64_t>(cntr, 1), s);
  nsel.alloc(1, s);
  NURI_CUDA(cudaMemsetAsync(nsel.p, 0, 4, s));
  if (cntr > 0) {
    ++launches;
    k_wselect<<<wgrid(cntr), 256, 0, s>>>(res.p, cntr, tau, g.vert_of, selV.p, selN.p, selS.p,
                                          nsel.p);
  }
  int32_t ns = 0;
  NURI_CUDA(cudaMemcpyAsync(&ns, nsel.p, 4, cudaMemcpyDeviceToHost, s));
  NURI_CUDA(cudaStreamSynchronize(s));
  DBuf<int32_t> perm, perm2;
  DBuf<uint32_t> key, key2;
  perm.alloc(std::max(ns, 1), s);
  perm2.alloc(std::max(ns, 1), s);
  key.alloc(std::max(ns, 1), s);
  key2.alloc(std::max(ns, 1), s);
  int maxc = 0;
  if (ns > 0) {
    DBuf<int32_t> mx;
    mx.alloc(1, s);
    NURI_CUDA(cudaMemsetAsync(mx.p, 0, 4, s));
    ++launches;
    k_wmax_rows<<<wgrid(ns), 256, 0, s>>>(selN.p, ns, mx.p);
    NURI_CUDA(cudaMemcpyAsync(&maxc, mx.p, 4, cudaMemcpyDeviceToHost, s));
    ++launches;
    k_wiota<<<wgrid(ns), 256, 0, s>>>(perm.p, ns);
    size_t tb = 0;
    cub::DeviceRadixSort::SortPairs(nullptr, tb, key.p, key2.p, perm.p, perm2.p, ns, 0, 32, s);
    DBuf<uint8_t> tmp;
    tmp.alloc(tb, s);
    NURI_CUDA(cudaStreamSynchronize(s));
    // least significant column first; the score's two words last (stable passes)
    for (int col = maxc - 1; col >= -2; --col) {
      ++launches;
      k_wcol<<<wgrid(ns), 256, 0, s>>>(selV.p, selN.p, selS.p, perm.p, ns, col, key.p);
      NURI_CUDA(cub::DeviceRadixSort::SortPairs(tmp.p, tb, key.p, key2.p, perm.p, perm2.p, ns,
                                                0, 32, s));
      std::swap(perm.p, perm2.p);
    }
  }
  // the rows ranked: the first k, or (NURI_KEEP_TIES) every row scoring at least the k-th.
  // tau may sit below the k-th score (coarse histogram bins), so the cut is made here.
  int32_t count = std::min(ns, k);
  if (keep_ties && ns > k) {
    std::vector<long long> scores(ns);
    DBuf<long long> sorted;
    sorted.alloc(ns, s);
    ++launches;
    k_wsorted_scores<<<wgrid(ns), 256, 0, s>>>(selS.p, perm.p, ns, sorted.p);
    NURI_CUDA(cudaMemcpyAsync(scores.data(), sorted.p, sizeof(long long) * ns,
                              cudaMemcpyDeviceToHost, s));
    NURI_CUDA(cudaStreamSynchronize(s));
    while (count < ns && scores[count] == scores[k - 1]) ++count;
  }
  std::vector<int32_t> sizes(std::max(count, 1));
  if (count > 0) {
    DBuf<int32_t> dsz;
    dsz.alloc(count, s);
    ++launches;
    k_wsizes<<<wgrid(count), 256, 0, s>>>(selN.p, perm.p, count, dsz.p);
    NURI_CUDA(cudaMemcpyAsync(sizes.data(), dsz.p, sizeof(int32_t) * count, cudaMemcpyDeviceToHost, s));
    NURI_CUDA(cudaStreamSynchronize(s));
  }
  int64_t nverts = 0;
  for (int i = 0; i < count; ++i) nverts += sizes[i];
  nuri_result* r = new_result(0, count, nverts, 0, false);
  r->vert_off[0] = 0;
  for (int i = 0; i < count; ++i) r->vert_off[i + 1] = r->vert_off[i] + sizes[i];
  for (int i = 0; i <= count; ++i) r->edge_off[i] = 0;
  if (count > 0) {
    DBuf<int32_t> dOff, dV;
    DBuf<long long> dS;
    dOff.alloc(count + 1, s);
    dV.alloc(std::max<int64_t>(nverts, 1), s);
    dS.alloc(count, s);
    NURI_CUDA(cudaMemcpyAsync(dOff.p, r->vert_off, sizeof(int32_t) * (count + 1),
                              cudaMemcpyHostToDevice, s));
    ++launches;
    k_wemit<<<wgrid(count), 256, 0, s>>>(selV.p, selN.p, selS.p, perm.p, count, dOff.p, dV.p,
                                         dS.p);
    NURI_CUDA(cudaMemcpyAsync(r->verts, dV.p, sizeof(int32_t) * nverts, cudaMemcpyDeviceToHost, s));
    NURI_CUDA(cudaMemcpyAsync(r->score, dS.p, sizeof(int64_t) * count, cudaMemcpyDeviceToHost, s));
    NURI_CUDA(cudaStreamSynchronize(s));
  }
  stats.expansions = (int64_t)hs.expansions;
  stats.pruned = (int64_t)hs.pruned;
  stats.dequeued = (int64_t)hs.dequeued;
  stats.adj_bytes = (int64_t)hs.adj_bytes;
  stats.results_stored = (int64_t)hs.res_count;
  stats.threshold = hs.tau == LLONG_MIN ? INT64_MIN : hs.tau;
  stats.restarts = restarts;
  stats.device_ms = timer.stop();
  stats.launches = launches;
  r->stats = stats;
  *out = r;
}

}  // namespace nuri
