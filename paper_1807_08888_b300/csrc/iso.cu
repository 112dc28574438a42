// Top-k labelled subgraph isomorphism: Algorithm 1 with the user functions of Section 4.3.
//
//   score(s)   = sum of the vertex scores of the matched data vertices (int32 weights, or
//                degrees as in the paper's evaluation)
//   u(s)       = sum over unmatched query vertices q of index(mu(root), label(q), hop(q)),
//                index = hop/label max index built at load time (Listing 3, cumulative hops);
//                hops beyond the resident index use the per-label global maximum
//   edge ranking (Section 2's cumulative edge weight): score(s) = sum of the weights of the
//                image's edges; u(s) = for every unmatched query edge, the heaviest edge its
//                images could use (from a matched image: that image's heaviest edge to the
//                other end's label; else the heaviest edge between the two labels)
//   dominated  = score + u < tau (strict), tau = k-th best score found so far (per query)
//   expandable = the added data vertex keeps the partial subgraph isomorphic to the matched
//                part of the query (label, injectivity, every query edge to a matched vertex)
//   results    = distinct image subgraphs (V_s, E_s): automorphic mappings are removed by
//                symmetry-breaking order constraints mu(a) < mu(b) derived from Aut(q)
//
// GPU organisation (one launch for a whole batch of queries):
//   * host: per query a breadth-first matching order from the minimum-eccentricity root,
//     the tree parent and hop of every position, back edges, and the symmetry-breaking
//     constraints (automorphisms by backtracking over <= 8! label-preserving permutations;
//     orbit-stabiliser chain);
//   * seeds (Algorithm 1, initialisation): every data vertex with the root's label, for every query, with
//     its bound score(v) + u; all seeds of all queries are sorted by bound, descending;
//   * k_iso_search: one warp per seed, dynamic assignment in bound order; the warp runs a
//     depth-first search over the matching order.  Candidates of a level come from the
//     label segment of the parent's image, which is sorted by score descending: the warp
//     evaluates 32 candidates per step (coalesced int2 loads; injectivity, symmetry and
//     back-edge binary searches per lane; ballot), descends into the valid ones in order,
//     and stops a level at the first candidate whose bound falls below tau (every later one
//     is smaller).  The last level writes its valid candidates as results directly.
//   * tau per query from a score histogram (16384 bins, exact for weight sums <= 16383),
//     scanned cooperatively by the warp that added results, published with atomicMax.
//   * top-k merge: rows with score >= tau of every query, keyed by (sorted vertex ids, sorted
//     edges), least-significant-column-first radix passes, then (query, score desc).
#include <cub/cub.cuh>

#include <algorithm>
#include <climits>
#include <cstdlib>
#include <cstring>
#include <functional>
#include <vector>

#include "nuri_internal.cuh"
#include "topk_common.cuh"

namespace nuri {
namespace {

constexpr int QMAX = 8;
constexpr int EMAX = 28;
constexpr int NBINS = 16384;
constexpr int ISO_WARPS = 8;
constexpr long long NONE = -(1ll << 50);

struct IsoQuery {
  int32_t nq, k;
  int32_t order[QMAX];   // query vertex at position i
  int32_t ppos[QMAX];    // position of the tree parent (i >= 1)
  int32_t hop[QMAX];     // hop (query distance from the root) of position i
  int32_t lab[QMAX];     // label of position i
  uint32_t back[QMAX];   // earlier positions adjacent to position i, parent excluded
  uint32_t nonadj[QMAX]; // induced matching: earlier positions NOT adjacent to position i
  uint32_t sym_lt[QMAX]; // earlier positions a that must satisfy mu(a) < mu(i)
  uint32_t sym_gt[QMAX]; // earlier positions a that must satisfy mu(a) > mu(i)
  int32_t ne;
  int32_t epos[EMAX][2]; // query edges as position pairs
  int32_t shift;         // histogram bin = score >> shift
  int32_t refine;        // bound each unmatched position by its nearest matched one
  int8_t qd[QMAX][QMAX]; // query distance between positions
};

struct IsoState {
  long long tau;                 // -1 while fewer than k results exist
  unsigned long long res_count;
  unsigned long long expansions, pruned, dequeued, bytes;
  int32_t hmax;                  // highest non-empty histogram bin
  int32_t err;
};

struct IsoRes {
  long long score;
  int32_t mu[QMAX];  // data vertex at each position
};

struct IsoCtx {
  DevGraph g;
  const int2* seg;          // weight- or degree-ranked label segments
  const int32_t* idx;       // hop index (nullptr when H == 0)
  const int32_t* gmax;      // per-label global maxima
  const int32_t* vscore;    // score of a vertex (weights or degrees; unused by edge ranking)
  const int32_t* ew;        // edge ranking: weight of every CSR entry
  const int32_t* emax;      // edge ranking: [n*L] heaviest edge from a vertex to a label
  const int32_t* lpmax;     // edge ranking: [L*L] heaviest edge between two labels
  int32_t edge;             // 1: rank by cumulative edge weight (seg = edge-weight segments)
  const IsoQuery* qs;
  IsoState* st;
  int32_t* hist;            // [nqueries][NBINS]
  IsoRes* res;
  const int64_t* res_base;  // first slot of each query's result region
  const int64_t* res_cap;   // capacity of each region
  const uint64_t* deadline;  // global timer value after which the search stops
  int32_t* err;              // bit 2: time budget exhausted
  unsigned long long* work_next;
};

__device__ __forceinline__ long long ld_volatile64(const long long* p) {
  return *(const volatile long long*)p;
}

__device__ __forceinline__ bool row_contains(const DevGraph& g, int32_t a, int32_t b) {
  // binary search of b in the id-sorted row of a (the shorter of the two rows is used)
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

// Edge ranking: the weight of the edge {a, b}, or -1 when a and b are not adjacent (the
// shorter row is searched; both directions of an edge carry its weight).
__device__ __forceinline__ int32_t row_weight(const IsoCtx& cx, int32_t a, int32_t b) {
  const DevGraph& g = cx.g;
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
  return lo < ea && __ldg(g.adj + lo) == x ? __ldg(cx.ew + lo) : -1;
}

// Edge ranking: an upper bound of the weights of the query edges from position p to the
// positions before it, when the positions below m are matched (images mu): an edge to a
// matched image weighs at most that image's heaviest edge to label(p), any other edge at most
// the heaviest edge between the two labels.  NONE when such an edge cannot exist.
__device__ __forceinline__ long long edge_bound(const IsoCtx& cx, const IsoQuery& Q,
                                                const int32_t* mu, int p, int m) {
  const int L = cx.g.L;
  uint32_t pred = Q.back[p] | (1u << Q.ppos[p]);
  long long t = 0;
  while (pred) {
    const int a = __ffs(pred) - 1;
    pred &= pred - 1;
    const int32_t x = a < m ? __ldg(cx.emax + (int64_t)mu[a] * L + Q.lab[p])
                            : __ldg(cx.lpmax + Q.lab[a] * L + Q.lab[p]);
    if (x < 0) return NONE;
    t += x;
  }
  return t;
}

__device__ __forceinline__ long long index_value(const IsoCtx& cx, int32_t v, int32_t hop,
                                                 int32_t lab) {
  if (cx.idx && hop <= cx.g.H)
    return __ldg(cx.idx + ((int64_t)(hop - 1) * cx.g.n + v) * cx.g.L + lab);
  return __ldg(cx.gmax + lab);
}

// Warp-cooperative threshold refresh for query q after results were added.
__device__ void refresh_tau(const IsoCtx& cx, int q, int64_t k, int32_t shift) {
  const int lane = threadIdx.x & 31;
  const int32_t* h = cx.hist + (int64_t)q * NBINS;
  IsoState* S = cx.st + q;
  // the loop below is warp-wide: its bounds must be the same in every lane
  const int32_t top = warp_load(&S->hmax);
  const long long tau = warp_load(&S->tau);
  int32_t floor_bin = tau < 0 ? 0 : (int32_t)(tau >> shift);
  long long acc = 0;
  for (int32_t b0 = top; b0 >= floor_bin; b0 -= 32) {
    int32_t b = b0 - lane;
    long long c = (b >= floor_bin) ? (long long)*(volatile const int32_t*)(h + b) : 0;
    // inclusive prefix from the top bin downwards
    long long x = c;
    for (int o = 1; o < 32; o <<= 1) {
      long long y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    long long tot = acc + x;
    unsigned hit = __ballot_sync(0xffffffffu, b >= floor_bin && tot >= k);
    if (hit) {
      int first = __ffs(hit) - 1;
      int32_t bin = b0 - first;
      long long t = (long long)bin << shift;
      if (lane == 0 && t > ld_volatile64(&S->tau)) atomicMax(&S->tau, t);
      return;
    }
    acc += __shfl_sync(0xffffffffu, x, 31);
  }
}

// Seeds: one per (query, vertex with the root's label); bound = score(v) + u.  With a seed
// partition, the roots of other parts get the bound NONE (never expanded).
__global__ void k_iso_seeds(IsoCtx cx, int32_t q, int64_t base, int64_t count, int32_t rootlab,
                            int32_t part_index, int32_t part_count, long long* keys,
                            unsigned long long* vals) {
  const IsoQuery Q = cx.qs[q];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x) {
    int32_t v = cx.g.lab_vert[cx.g.lab_off[rootlab] + i];
    vals[base + i] = ((unsigned long long)(uint32_t)q << 32) | (uint32_t)v;
    if (part_count > 1 && seed_part(v, part_count) != part_index) {
      keys[base + i] = NONE;
      continue;
    }
    long long b = cx.edge ? 0 : __ldg(cx.vscore + v);
    for (int p = 1; p < Q.nq; ++p) {
      long long x = cx.edge ? edge_bound(cx, Q, &v, p, 1) : index_value(cx, v, Q.hop[p], Q.lab[p]);
      if (x < 0) {
        b = NONE;
        break;
      }
      b += x;
    }
    keys[base + i] = b;
  }
}

// Items of the search: a seed (query q, root image v) whose first-level candidate list (the
// root's segment for the label of query position 1) is long is split into chunks of
// kSeedChunk candidates, one item each, so that a hub root does not leave one warp working
// long after the others (the search is tail-bound otherwise).  Every match is found once,
// in the chunk holding its position-1 image.  An item's key is a bound for its chunk: the
// root's score, the chunk's first (largest) candidate score, and the index bound of the
// positions after 1.  Encoding: q << kItemQShift | chunk << 31 | v.
constexpr int kSeedChunk = 64;
constexpr int kItemQShift = 52;
constexpr unsigned long long kItemChunkMask = (1ull << (kItemQShift - 31)) - 1;

__global__ void k_iso_chunk_count(IsoCtx cx, const long long* __restrict__ keys,
                                  const unsigned long long* __restrict__ vals, int64_t n,
                                  int64_t* __restrict__ cnt) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int q = (int)(vals[i] >> 32);
    const int32_t v = (int32_t)(uint32_t)vals[i];
    const IsoQuery& Q = cx.qs[q];
    int64_t c = 1;
    if (keys[i] != NONE && Q.nq > 1) {
      const int64_t so = (int64_t)v * cx.g.L + Q.lab[1];
      const int64_t len = cx.g.lsoff[so + 1] - cx.g.lsoff[so];
      c = len > kSeedChunk ? (len + kSeedChunk - 1) / kSeedChunk : 1;
      if (c > (int64_t)kItemChunkMask + 1) c = (int64_t)kItemChunkMask + 1;  // unreachable
    }
    cnt[i] = c;
  }
}

__global__ void k_iso_chunk_write(IsoCtx cx, const long long* __restrict__ keys,
                                  const unsigned long long* __restrict__ vals, int64_t n,
                                  const int64_t* __restrict__ off, long long* __restrict__ okeys,
                                  unsigned long long* __restrict__ ovals) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const unsigned long long q = vals[i] >> 32;
    const int32_t v = (int32_t)(uint32_t)vals[i];
    const IsoQuery& Q = cx.qs[q];
    const int64_t o = off[i], c = off[i + 1] - off[i];
    for (int64_t j = 0; j < c; ++j) {
      long long key = keys[i];
      if (key != NONE && Q.nq > 1) {
        const int64_t so = (int64_t)v * cx.g.L + Q.lab[1];
        const int64_t at = cx.g.lsoff[so] + j * kSeedChunk;
        if (at < cx.g.lsoff[so + 1]) {
          // replace position 1's bound by the chunk's largest candidate score (edge ranking:
          // the weight of the chunk's heaviest edge from the root; position 1 has no other
          // edge to an earlier position)
          const long long first =
              cx.edge ? (long long)__ldg(cx.emax + (int64_t)v * cx.g.L + Q.lab[1])
                      : index_value(cx, v, Q.hop[1], Q.lab[1]);
          key = key - first + (long long)__ldg(cx.seg + at).y;
        } else {
          key = NONE;  // an empty segment: the item finds nothing
        }
      }
      okeys[o + j] = key;
      ovals[o + j] = (q << kItemQShift) | ((unsigned long long)j << 31) | (unsigned)v;
    }
  }
}

// Raise query q's threshold to at least v (published by another part of a partitioned run).
__global__ void k_iso_raise_tau(IsoState* st, int32_t q, long long v) {
  if (threadIdx.x == 0 && blockIdx.x == 0) atomicMax(&st[q].tau, v);
}

__device__ void add_results_leaf(const IsoCtx& cx, int q, const IsoQuery& Q, bool valid,
                                 long long score, const int32_t* mu, int32_t last) {
  const int lane = threadIdx.x & 31;
  unsigned m = __ballot_sync(0xffffffffu, valid);
  if (!m) return;
  IsoState* S = cx.st + q;
  if (valid) {
    unsigned long long slot = atomicAdd(&S->res_count, 1ull);
    if ((int64_t)slot < cx.res_cap[q]) {
      IsoRes* r = cx.res + cx.res_base[q] + slot;
      r->score = score;
      for (int i = 0; i < Q.nq - 1; ++i) r->mu[i] = mu[i];
      r->mu[Q.nq - 1] = last;
    }
    long long bl = score >> Q.shift;
    int32_t bin = bl >= NBINS ? NBINS - 1 : (int32_t)bl;
    atomicAdd(cx.hist + (int64_t)q * NBINS + bin, 1);
    if (bin > *(volatile int32_t*)&S->hmax) atomicMax(&S->hmax, bin);
  }
  __syncwarp();
  __threadfence_block();
  // tau stays "none" until k results exist
  if ((int64_t)warp_load(&S->res_count) < (int64_t)Q.k) return;
  refresh_tau(cx, q, Q.k, Q.shift);
  (void)lane;
}

__global__ void __launch_bounds__(ISO_WARPS * 32) k_iso_search(IsoCtx cx,
                                                               const long long* __restrict__ keys,
                                                               const unsigned long long* __restrict__ vals,
                                                               int64_t nitems) {
  const int lane = threadIdx.x & 31;
  const unsigned FULL = 0xffffffffu;
  const DevGraph& g = cx.g;
  unsigned long long my_exp = 0, my_pruned = 0, my_deq = 0, my_bytes = 0;
  while (true) {
    int64_t item = 0;
    if (lane == 0) {
      item = (int64_t)atomicAdd(cx.work_next, 1ull);
      if (item < nitems && global_ns() > *(const volatile uint64_t*)cx.deadline) {
        atomicOr(cx.err, 4);
        item = nitems;
      }
    }
    item = __shfl_sync(FULL, item, 0);
    if (item >= nitems) break;
    long long bound = keys[item];
    unsigned long long pv = vals[item];
    int q = (int)(pv >> kItemQShift);
    int32_t v = (int32_t)(pv & 0x7FFFFFFFull);
    const int64_t chunk = (int64_t)((pv >> 31) & kItemChunkMask);
    IsoState* S = cx.st + q;
    long long tau = warp_load(&S->tau);
    if (bound == NONE || bound < tau) {
      if (lane == 0) ++my_pruned;
      continue;
    }
    const IsoQuery& Q = cx.qs[q];
    const int nq = Q.nq;
    if (lane == 0) ++my_deq;
    // rest[i] = sum over positions > i of the index bound (fixed by the root image).  Edge
    // ranking: rest[i] bounds the edges of the positions after i, bk[i] the back edges of
    // position i itself (both set when position i is reached, from the images matched then)
    long long rest[QMAX], bk[QMAX], sx[QMAX];
    int32_t mu[QMAX];
    long long sc[QMAX + 1];
    mu[0] = v;
    if (cx.edge) {
      long long acc = 0;
      for (int p = 2; p < nq; ++p) {
        const long long x = edge_bound(cx, Q, mu, p, 1);
        acc = (x < 0 || acc < 0) ? NONE : acc + x;
      }
      rest[1] = acc;
      bk[1] = 0;  // position 1's only earlier position is its parent
      sc[1] = 0;
    } else {
      long long acc = 0;
      for (int p = nq - 1; p >= 0; --p) {
        rest[p] = acc;
        if (p >= 1) acc += index_value(cx, v, Q.hop[p], Q.lab[p]);
      }
      sc[1] = __ldg(cx.vscore + v);
    }
    if (nq == 1) {
      // the seed is a complete match
      bool valid = lane == 0 && sc[1] >= tau;
      add_results_leaf(cx, q, Q, valid, sc[1], mu, v);
      continue;
    }
    int64_t pos[QMAX], end[QMAX], base[QMAX];
    unsigned mask[QMAX];
    int lev = 1;
    {
      // this item's chunk of the first level's candidates (the root's label segment)
      int32_t a = mu[Q.ppos[1]];
      int64_t so = (int64_t)a * g.L + Q.lab[1];
      pos[1] = g.lsoff[so] + chunk * kSeedChunk;
      end[1] = min(g.lsoff[so + 1], pos[1] + (int64_t)kSeedChunk);
      mask[1] = 0;
    }
    unsigned steps = 0;
    while (lev >= 1) {
      if (mask[lev] == 0) {
        if (pos[lev] >= end[lev]) {
          --lev;
          continue;
        }
        if ((++steps & 255) == 0 && warp_past(cx.deadline)) {
          if (lane == 0) atomicOr(cx.err, 4);
          break;
        }
        tau = warp_load(&S->tau);
        int64_t i = pos[lev] + lane;
        bool in = i < end[lev];
        int2 c = in ? __ldg(cx.seg + i) : make_int2(-1, -1);
        long long s_new = sc[lev] + (long long)c.y;
        // candidates come in descending c.y: this bound falls along the segment
        bool okb = in && (s_new + (cx.edge ? bk[lev] : 0) + rest[lev] >= tau);
        bool valid = okb;
        if (valid)
          for (int a = 0; a < lev; ++a)
            if (mu[a] == c.x) valid = false;
        if (valid) {
          uint32_t m = Q.sym_lt[lev];
          while (m && valid) {
            int a = __ffs(m) - 1;
            m &= m - 1;
            if (!(mu[a] < c.x)) valid = false;
          }
          m = Q.sym_gt[lev];
          while (m && valid) {
            int a = __ffs(m) - 1;
            m &= m - 1;
            if (!(mu[a] > c.x)) valid = false;
          }
        }
        if (valid) {
          uint32_t m = Q.back[lev];
          while (m && valid) {
            int a = __ffs(m) - 1;
            m &= m - 1;
            if (cx.edge) {  // the back edge's weight joins the score
              const int32_t wb = row_weight(cx, mu[a], c.x);
              valid = wb >= 0;
              s_new += wb;
            } else {
              valid = row_contains(g, mu[a], c.x);
            }
          }
          // induced matching: no data edge where the query has none
          m = Q.nonadj[lev];
          while (m && valid) {
            int a = __ffs(m) - 1;
            m &= m - 1;
            valid = !row_contains(g, mu[a], c.x);
          }
        }
        if (cx.edge) {
          // the exact score (tree and back edges) against tau; kept for the descent
          if (valid && s_new + rest[lev] < tau) valid = false;
          sx[lev] = s_new;
        }
        unsigned inm = __ballot_sync(FULL, in);
        unsigned okm = __ballot_sync(FULL, okb);
        unsigned vm = __ballot_sync(FULL, valid);
        if (lane == 0) {
          my_exp += __popc(vm);
          my_pruned += __popc(inm & ~okm);
          my_bytes += 8ull * __popc(inm);
        }
        base[lev] = pos[lev];
        // candidates are sorted by score: the first failing bound ends the level
        if ((inm & ~okm) != 0) pos[lev] = end[lev];
        else pos[lev] += 32;
        if (lev == nq - 1) {
          add_results_leaf(cx, q, Q, valid, s_new, mu, c.x);
          continue;
        }
        mask[lev] = vm;
        continue;
      }
      // descend into the next valid candidate of this level
      int b = __ffs(mask[lev]) - 1;
      mask[lev] &= mask[lev] - 1;
      int2 c = __ldg(cx.seg + base[lev] + b);
      long long s_new = sc[lev] + (long long)c.y;
      long long s_exact = 0;  // edge ranking: the candidate's exact score, from its lane
      if (cx.edge) s_exact = __shfl_sync(FULL, sx[lev], b);
      tau = warp_load(&S->tau);
      if (s_new + (cx.edge ? bk[lev] : 0) + rest[lev] < tau) {
        // tau rose: this and every later candidate fail
        mask[lev] = 0;
        pos[lev] = end[lev];
        continue;
      }
      if (cx.edge) {
        if (s_exact + rest[lev] < tau) continue;  // this candidate only
        s_new = s_exact;
      }
      mu[lev] = c.x;
      sc[lev + 1] = s_new;
      ++lev;
      if (cx.edge) {
        // bounds of the new level from the images matched so far (positions < lev): lane p
        // takes the edges of position p > lev
        long long term = 0;
        if (lane > lev && lane < nq) term = edge_bound(cx, Q, mu, lane, lev);
        const bool none = __any_sync(FULL, term < 0);
        for (int o = 16; o; o >>= 1) term += __shfl_xor_sync(FULL, term, o);
        rest[lev] = none ? NONE : term;
        long long kb = 0;
        uint32_t m = Q.back[lev];
        while (m) {
          const int a = __ffs(m) - 1;
          m &= m - 1;
          const int32_t x = __ldg(cx.emax + (int64_t)mu[a] * g.L + Q.lab[lev]);
          if (x < 0) {
            kb = NONE;
            break;
          }
          kb += x;
        }
        bk[lev] = kb;
      } else if (Q.refine && lev + 1 < nq) {
        // rest[lev] = sum over the positions after lev of the smallest index bound any
        // matched position gives (each is a valid bound: the image lies within the query
        // distance, as a walk, of that matched image); lane p computes position p
        long long term = 0;
        if (lane > lev && lane < nq) {
          long long best = LLONG_MAX;
          for (int a = 0; a < lev; ++a)
            best = min(best, index_value(cx, mu[a], Q.qd[a][lane], Q.lab[lane]));
          term = best < 0 ? NONE : best;
        }
        for (int o = 16; o; o >>= 1) term += __shfl_xor_sync(FULL, term, o);
        rest[lev] = term < 0 ? NONE : term;  // matched position 0 is in the min: <= root bound
      }
      int32_t a = mu[Q.ppos[lev]];
      int64_t so = (int64_t)a * g.L + Q.lab[lev];
      pos[lev] = g.lsoff[so];
      end[lev] = g.lsoff[so + 1];
      mask[lev] = 0;
    }
  }
  if (lane == 0) {
    // counters of this warp go to query 0's slot only as totals (summed on the host)
    atomicAdd(&cx.st[0].expansions, my_exp);
    atomicAdd(&cx.st[0].pruned, my_pruned);
    atomicAdd(&cx.st[0].dequeued, my_deq);
    atomicAdd(&cx.st[0].bytes, my_bytes);
  }
}

// ---- top-k merge ----
constexpr int KCOLS = QMAX + 2 * EMAX;  // sorted vertex ids, then sorted edge endpoints

__global__ void k_iso_select(IsoCtx cx, int32_t nqueries, const long long* taus,
                             const int64_t* counts, int32_t* sel_q, long long* sel_score,
                             int32_t* sel_key, int32_t* nsel) {
  // one thread per stored result of every query
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int q = 0; q < nqueries; ++q) {
    int64_t cnt = counts[q];
    const IsoQuery& Q = cx.qs[q];
    for (int64_t i = t; i < cnt; i += stride) {
      const IsoRes& r = cx.res[cx.res_base[q] + i];
      if (r.score < taus[q]) continue;
      int pos = atomicAdd(nsel, 1);
      sel_q[pos] = q;
      sel_score[pos] = r.score;
      int32_t* key = sel_key + (int64_t)pos * KCOLS;
      int32_t V[QMAX];
      for (int a = 0; a < Q.nq; ++a) V[a] = r.mu[a];
      for (int a = 1; a < Q.nq; ++a) {
        int32_t x = V[a];
        int b = a - 1;
        while (b >= 0 && V[b] > x) {
          V[b + 1] = V[b];
          --b;
        }
        V[b + 1] = x;
      }
      for (int a = 0; a < QMAX; ++a) key[a] = a < Q.nq ? V[a] : -1;
      long long E[EMAX];
      for (int e = 0; e < Q.ne; ++e) {
        int32_t x = r.mu[Q.epos[e][0]], y = r.mu[Q.epos[e][1]];
        int32_t lo = min(x, y), hi = max(x, y);
        E[e] = ((long long)lo << 32) | (unsigned)hi;
      }
      for (int a = 1; a < Q.ne; ++a) {
        long long x = E[a];
        int b = a - 1;
        while (b >= 0 && E[b] > x) {
          E[b + 1] = E[b];
          --b;
        }
        E[b + 1] = x;
      }
      for (int e = 0; e < EMAX; ++e) {
        key[QMAX + 2 * e] = e < Q.ne ? (int32_t)(E[e] >> 32) : -1;
        key[QMAX + 2 * e + 1] = e < Q.ne ? (int32_t)(uint32_t)E[e] : -1;
      }
    }
  }
}

__global__ void k_iso_col(const int32_t* key, const int32_t* perm, int32_t n, int col,
                          uint32_t* out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (uint32_t)(key[(int64_t)perm[i] * KCOLS + col] + 1);
}

__global__ void k_iso_final_key(const int32_t* sel_q, const long long* sel_score,
                                const int32_t* perm, int32_t n, unsigned long long* out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    int32_t r = perm[i];
    // (query asc, score desc); scores < 2^48
    out[i] = ((unsigned long long)sel_q[r] << 48) |
             ((1ull << 48) - 1 - (unsigned long long)sel_score[r]);
  }
}

__global__ void k_iota32(int32_t* a, int32_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    a[i] = (int32_t)i;
}

inline int gridn(int64_t n) {
  int64_t b = (n + 255) / 256;
  return (int)std::max<int64_t>(1, std::min<int64_t>(b, 1 << 20));
}

// ---- host-side query preparation ----
struct Prepared {
  IsoQuery q;
  int32_t rootlab;
  int64_t maxscore;
  bool empty;  // a query label absent from the data graph: no match exists
};

bool prepare_query(const nuri_query& in, int32_t k, const std::vector<int32_t>& gmax, int L,
                   bool induced, Prepared* out) {
  int nq = in.nq;
  int A[QMAX][QMAX] = {};
  for (int e = 0; e < in.ne; ++e) {
    int a = in.src[e], b = in.dst[e];
    if (a < 0 || b < 0 || a >= nq || b >= nq || a == b) return false;
    A[a][b] = A[b][a] = 1;
  }
  out->empty = false;
  for (int i = 0; i < nq; ++i)
    if (in.labels[i] >= L) out->empty = true;  // valid query, but no match can exist
  auto bfs = [&](int r, int* dist, int* order, int* par) {
    for (int i = 0; i < nq; ++i) dist[i] = -1, par[i] = -1;
    int head = 0, tail = 0;
    order[tail++] = r;
    dist[r] = 0;
    while (head < tail) {
      int a = order[head++];
      for (int b = 0; b < nq; ++b)
        if (A[a][b] && dist[b] < 0) {
          dist[b] = dist[a] + 1;
          par[b] = a;
          order[tail++] = b;
        }
    }
    return tail;
  };
  int dist[QMAX], order[QMAX], par[QMAX];
  int root = -1, best = 1 << 30;
  for (int r = 0; r < nq; ++r) {
    if (bfs(r, dist, order, par) != nq) return false;  // disconnected
    int ecc = 0;
    for (int i = 0; i < nq; ++i) ecc = std::max(ecc, dist[i]);
    if (ecc < best) {
      best = ecc;
      root = r;
    }
  }
  bfs(root, dist, order, par);
  IsoQuery& Q = out->q;
  memset(&Q, 0, sizeof(Q));
  Q.nq = nq;
  Q.k = k;
  int posof[QMAX];
  for (int i = 0; i < nq; ++i) {
    Q.order[i] = order[i];
    posof[order[i]] = i;
  }
  for (int i = 0; i < nq; ++i) {
    int qv = order[i];
    Q.hop[i] = dist[qv];
    Q.lab[i] = in.labels[qv];
    Q.ppos[i] = i == 0 ? -1 : posof[par[qv]];
    uint32_t bk = 0, na = 0;
    for (int j = 0; j < i; ++j) {
      if (A[qv][order[j]] && j != Q.ppos[i]) bk |= 1u << j;
      if (!A[qv][order[j]]) na |= 1u << j;
    }
    Q.back[i] = bk;
    Q.nonadj[i] = induced ? na : 0u;
  }
  Q.ne = 0;
  for (int a = 0; a < nq; ++a)
    for (int b = a + 1; b < nq; ++b)
      if (A[a][b]) {
        Q.epos[Q.ne][0] = posof[a];
        Q.epos[Q.ne][1] = posof[b];
        ++Q.ne;
      }
  // automorphisms (label- and edge-preserving permutations)
  std::vector<std::vector<int>> aut;
  {
    std::vector<int> perm(nq, -1);
    std::vector<char> used(nq, 0);
    std::function<void(int)> rec = [&](int i) {
      if (i == nq) {
        aut.push_back(perm);
        return;
      }
      for (int c = 0; c < nq; ++c) {
        if (used[c] || in.labels[c] != in.labels[i]) continue;
        bool ok = true;
        for (int j = 0; j < i && ok; ++j)
          if (A[i][j] != A[c][perm[j]]) ok = false;
        if (!ok) continue;
        used[c] = 1;
        perm[i] = c;
        rec(i + 1);
        used[c] = 0;
        perm[i] = -1;
      }
    };
    rec(0);
  }
  // symmetry breaking: orbit-stabiliser chain; constraint mu(v) < mu(w) per orbit member
  while (aut.size() > 1) {
    int pick = -1;
    std::vector<int> orb;
    for (int v = 0; v < nq && pick < 0; ++v) {
      std::vector<int> o;
      for (auto& s : aut)
        if (std::find(o.begin(), o.end(), s[v]) == o.end()) o.push_back(s[v]);
      if (o.size() > 1) {
        pick = v;
        orb = o;
      }
    }
    if (pick < 0) break;
    for (int w : orb) {
      if (w == pick) continue;
      int pv = posof[pick], pw = posof[w];
      if (pv < pw) Q.sym_lt[pw] |= 1u << pv;   // mu(pick) < mu(w), w matched later
      else Q.sym_gt[pv] |= 1u << pw;           // mu(w) > mu(pick), pick matched later
    }
    std::vector<std::vector<int>> stab;
    for (auto& s : aut)
      if (s[pick] == pick) stab.push_back(s);
    aut.swap(stab);
  }
  // query distances between positions (Floyd-Warshall on <= 8 vertices)
  {
    int D[QMAX][QMAX];
    for (int a = 0; a < nq; ++a)
      for (int b = 0; b < nq; ++b) D[a][b] = a == b ? 0 : (A[a][b] ? 1 : 64);
    for (int c = 0; c < nq; ++c)
      for (int a = 0; a < nq; ++a)
        for (int b = 0; b < nq; ++b) D[a][b] = std::min(D[a][b], D[a][c] + D[c][b]);
    for (int i = 0; i < nq; ++i)
      for (int j = 0; j < nq; ++j) Q.qd[i][j] = (int8_t)D[order[i]][order[j]];
  }
  Q.refine = getenv("NURI_ISO_ROOT_BOUND") ? 0 : 1;
  // histogram resolution: exact bins when every score fits
  int64_t mx = 0;
  for (int i = 0; i < nq; ++i) mx += in.labels[i] < L ? std::max(0, gmax[in.labels[i]]) : 0;
  int shift = 0;
  while ((mx >> shift) >= NBINS) ++shift;
  Q.shift = shift;
  out->rootlab = in.labels[order[0]];
  out->maxscore = mx;
  return true;
}

}  // namespace

// Upper bound of the device memory one isomorphism query with result size k allocates on
// graph G: its seeds (a whole label class at most) with their sort, its share of the batch
// state, its result region and the final selection and merge over that region.
int64_t iso_query_bytes(const nuri_graph* G, int32_t k) {
  const int64_t seeds = std::max<int64_t>(G->d.n, 1);
  const int64_t chunks = seeds + G->d.nnz / kSeedChunk;  // seeds split into first-level chunks
  const int64_t cap = std::max<int64_t>(65536, (int64_t)k * 256);  // the edge ranking's
  return seeds * (2 * 8 + 2 * 8 + 16) + chunks * (4 * 8 + 16) + (int64_t)NBINS * 4 +
         (int64_t)sizeof(IsoState) +
         (int64_t)sizeof(IsoQuery) +
         cap * ((int64_t)sizeof(IsoRes) + 4 + 8 + 4 * KCOLS + 4 * 4 + 8 * 2);
}

void topk_iso_batch(nuri_graph* G, int32_t nqueries, const nuri_query* qs, const int32_t* ks,
                    int32_t rank, uint32_t flags, cudaStream_t s, nuri_result** outs) {
  const DevGraph& g = G->d;
  DevTimer timer(s);
  const bool deg = rank == NURI_RANK_DEGREE_SUM;
  const bool edge = rank == NURI_RANK_EDGE_WEIGHT_SUM;
  const bool keep_ties = flags & NURI_KEEP_TIES;
  if (edge && !g.ew) NURI_FAIL(NURI_ERR_INVALID, "nuri_topk_iso: graph has no edge weights");
  if (rank == NURI_RANK_WEIGHT_SUM && !g.weights)
    NURI_FAIL(NURI_ERR_INVALID, "nuri_topk_iso: graph has no weights");
  const std::vector<int32_t> no_vertex_scores(std::max(g.L, 1), 0);
  const std::vector<int32_t>& gmax =
      edge ? no_vertex_scores : (deg ? G->h_gmax_d : G->h_gmax_w);
  int64_t launches = 0;
  if (nqueries >= (1 << (64 - kItemQShift)))
    NURI_FAIL(NURI_ERR_LIMIT, "nuri_topk_iso: at most %d queries in one batch",
              (1 << (64 - kItemQShift)) - 1);
  std::vector<Prepared> prep(nqueries);
  for (int i = 0; i < nqueries; ++i)
    if (!prepare_query(qs[i], ks[i], gmax, g.L, (flags & NURI_ISO_INDUCED) != 0, &prep[i]))
      NURI_FAIL(NURI_ERR_INVALID, "nuri_topk_iso: query %d is not a connected simple graph", i);
  if (edge)
    for (auto& pq : prep) {
      // histogram resolution from the largest edge-weight sum a match can have
      const int64_t mx = (int64_t)pq.q.ne * std::max(G->h_ewmax, 0);
      int shift = 0;
      while ((mx >> shift) >= NBINS) ++shift;
      pq.q.shift = shift;
      pq.maxscore = mx;
    }

  DBuf<IsoQuery> dq;
  dq.alloc(nqueries, s);
  {
    std::vector<IsoQuery> hq(nqueries);
    for (int i = 0; i < nqueries; ++i) hq[i] = prep[i].q;
    NURI_CUDA(cudaMemcpyAsync(dq.p, hq.data(), sizeof(IsoQuery) * nqueries, cudaMemcpyHostToDevice, s));
    NURI_CUDA(cudaStreamSynchronize(s));
  }
  // seeds of every query
  std::vector<int64_t> seed_base(nqueries + 1, 0);
  for (int i = 0; i < nqueries; ++i) {
    int rl = prep[i].rootlab;
    int64_t c = (!prep[i].empty && rl < g.L) ? G->h_lab_off[rl + 1] - G->h_lab_off[rl] : 0;
    seed_base[i + 1] = seed_base[i] + c;
  }
  int64_t nitems = seed_base[nqueries];

  IsoCtx cx;
  memset(&cx, 0, sizeof(cx));
  cx.g = g;
  cx.seg = edge ? g.lseg_e : (deg ? g.lseg_d : g.lseg_w);
  cx.idx = edge ? nullptr : (deg ? g.idx_d : g.idx_w);
  cx.gmax = edge ? nullptr : (deg ? g.gmax_d : g.gmax_w);
  cx.vscore = edge ? nullptr : (deg ? g.deg : g.weights);
  cx.ew = g.ew;
  cx.emax = g.emax;
  cx.lpmax = g.lpmax;
  cx.edge = edge ? 1 : 0;
  cx.qs = dq.p;

  DBuf<long long> keys, keys2;
  DBuf<unsigned long long> vals, vals2;
  keys.alloc(std::max<int64_t>(nitems, 1), s);
  keys2.alloc(std::max<int64_t>(nitems, 1), s);
  vals.alloc(std::max<int64_t>(nitems, 1), s);
  vals2.alloc(std::max<int64_t>(nitems, 1), s);
  for (int i = 0; i < nqueries; ++i) {
    int64_t c = seed_base[i + 1] - seed_base[i];
    if (c > 0) {
      ++launches;
      k_iso_seeds<<<gridn(c), 256, 0, s>>>(cx, i, seed_base[i], c, prep[i].rootlab,
                                           G->part.index, G->part.count, keys.p, vals.p);
    }
  }
  if (nitems > 0) {
    // split long first levels into chunks (see k_iso_chunk_count)
    DBuf<int64_t> ccnt, coff;
    ccnt.alloc(nitems + 1, s);
    coff.alloc(nitems + 1, s);
    NURI_CUDA(cudaMemsetAsync(ccnt.p + nitems, 0, sizeof(int64_t), s));
    ++launches;
    k_iso_chunk_count<<<gridn(nitems), 256, 0, s>>>(cx, keys.p, vals.p, nitems, ccnt.p);
    size_t tbs = 0;
    cub::DeviceScan::ExclusiveSum(nullptr, tbs, ccnt.p, coff.p, nitems + 1, s);
    DBuf<uint8_t> stmp;
    stmp.alloc(tbs, s);
    NURI_CUDA(cub::DeviceScan::ExclusiveSum(stmp.p, tbs, ccnt.p, coff.p, nitems + 1, s));
    int64_t nchunks = 0;
    NURI_CUDA(cudaMemcpyAsync(&nchunks, coff.p + nitems, 8, cudaMemcpyDeviceToHost, s));
    NURI_CUDA(cudaStreamSynchronize(s));
    DBuf<long long> ckeys;
    DBuf<unsigned long long> cvals;
    ckeys.alloc(std::max<int64_t>(nchunks, 1), s);
    cvals.alloc(std::max<int64_t>(nchunks, 1), s);
    ++launches;
    k_iso_chunk_write<<<gridn(nitems), 256, 0, s>>>(cx, keys.p, vals.p, nitems, coff.p, ckeys.p,
                                                   cvals.p);
    NURI_CUDA(cudaGetLastError());
    nitems = nchunks;
    keys = std::move(ckeys);
    vals = std::move(cvals);
    keys2.alloc(std::max<int64_t>(nitems, 1), s);
    vals2.alloc(std::max<int64_t>(nitems, 1), s);
    size_t tb = 0;
    cub::DeviceRadixSort::SortPairsDescending(nullptr, tb, keys.p, keys2.p, vals.p, vals2.p, nitems, 0, 64, s);
    DBuf<uint8_t> tmp;
    tmp.alloc(tb, s);
    NURI_CUDA(cub::DeviceRadixSort::SortPairsDescending(tmp.p, tb, keys.p, keys2.p, vals.p, vals2.p, nitems, 0, 64, s));
  }

  // per-query state, histograms, result regions
  std::vector<long long> tau_init(nqueries, -1);
  std::vector<int64_t> cap(nqueries), rbase(nqueries + 1);
  // result rows per query (40 B each): room for the rows recorded while tau is still low, so
  // that an overflow (which re-runs the batch) stays rare
  // (ranked by edge weight: four times that -- its looser bounds keep tau lower longer)
  for (int i = 0; i < nqueries; ++i)
    cap[i] = std::max<int64_t>(edge ? 65536 : 16384, (int64_t)ks[i] * (edge ? 256 : 64));
  if (const char* e = getenv("NURI_RESULT_CAP"))
    for (int i = 0; i < nqueries; ++i) cap[i] = std::max<int64_t>(1, atoll(e));
  std::vector<char> active(nqueries, 1);
  DBuf<IsoState> st;
  st.alloc(nqueries, s);
  DBuf<int32_t> hist;
  hist.alloc((int64_t)nqueries * NBINS, s);
  DBuf<int64_t> d_rbase, d_cap;
  d_rbase.alloc(nqueries, s);
  d_cap.alloc(nqueries, s);
  DBuf<unsigned long long> work;
  work.alloc(1, s);
  DBuf<uint64_t> deadline;
  deadline.alloc(1, s);
  DBuf<int32_t> derr;
  derr.alloc(1, s);
  NURI_CUDA(cudaMemsetAsync(derr.p, 0, 4, s));
  ++launches;
  k_set_deadline<<<1, 32, 0, s>>>(deadline.p, time_budget_ns());
  cx.deadline = deadline.p;
  cx.err = derr.p;
  DBuf<IsoRes> res;
  std::vector<IsoState> hs(nqueries);
  nuri_stats total;
  memset(&total, 0, sizeof(total));
  int restarts = 0;
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

  // results that are final per query (kept across re-runs)
  std::vector<IsoState> final_state(nqueries);
  DBuf<IsoRes> final_res;  // not used: selection happens after the last pass
  while (true) {
    rbase[0] = 0;
    for (int i = 0; i < nqueries; ++i) rbase[i + 1] = rbase[i] + (active[i] ? cap[i] : 0);
    res.alloc(std::max<int64_t>(rbase[nqueries], 1), s);
    std::vector<IsoState> init(nqueries);
    memset(init.data(), 0, sizeof(IsoState) * nqueries);
    for (int i = 0; i < nqueries; ++i) {
      init[i].tau = active[i] ? tau_init[i] : LLONG_MAX;  // inactive queries prune everything
      init[i].hmax = 0;
    }
    NURI_CUDA(cudaMemcpyAsync(st.p, init.data(), sizeof(IsoState) * nqueries, cudaMemcpyHostToDevice, s));
    NURI_CUDA(cudaMemsetAsync(hist.p, 0, sizeof(int32_t) * nqueries * NBINS, s));
    NURI_CUDA(cudaMemcpyAsync(d_rbase.p, rbase.data(), sizeof(int64_t) * nqueries, cudaMemcpyHostToDevice, s));
    NURI_CUDA(cudaMemcpyAsync(d_cap.p, cap.data(), sizeof(int64_t) * nqueries, cudaMemcpyHostToDevice, s));
    NURI_CUDA(cudaMemsetAsync(work.p, 0, sizeof(unsigned long long), s));
    cx.st = st.p;
    cx.hist = hist.p;
    cx.res = res.p;
    cx.res_base = d_rbase.p;
    cx.res_cap = d_cap.p;
    cx.work_next = work.p;
    NURI_CUDA(cudaEventRecord(ev0, s));
    if (nitems > 0 && G->part.count > 1 && G->part.exchange) {
      // partitioned: the seeds in eight chunks (best bounds first), with the thresholds of
      // all parts exchanged between chunks
      const int64_t chunk = std::max<int64_t>((nitems + 7) / 8, 1 << 12);
      for (int64_t off = 0; off < nitems; off += chunk) {
        const int64_t cn = std::min(chunk, nitems - off);
        NURI_CUDA(cudaMemsetAsync(work.p, 0, sizeof(unsigned long long), s));
        ++launches;
        k_iso_search<<<sm_count() * 4, ISO_WARPS * 32, 0, s>>>(cx, keys2.p + off, vals2.p + off, cn);
        NURI_CUDA(cudaGetLastError());
        NURI_CUDA(cudaMemcpyAsync(hs.data(), st.p, sizeof(IsoState) * nqueries,
                                  cudaMemcpyDeviceToHost, s));
        NURI_CUDA(cudaStreamSynchronize(s));
        for (int i = 0; i < nqueries; ++i) {
          if (!active[i]) continue;
          const int64_t loc = hs[i].tau < 0 ? INT64_MIN : (int64_t)hs[i].tau;
          const int64_t glob = G->part.exchange(G->part.ctx, i, loc);
          if (glob > loc) {
            ++launches;
            k_iso_raise_tau<<<1, 32, 0, s>>>(st.p, i, (long long)glob);
          }
        }
      }
    } else if (nitems > 0) {
      ++launches;
      k_iso_search<<<sm_count() * 4, ISO_WARPS * 32, 0, s>>>(cx, keys2.p, vals2.p, nitems);
    }
    NURI_CUDA(cudaEventRecord(ev1, s));
    NURI_CUDA(cudaGetLastError());
    NURI_CUDA(cudaMemcpyAsync(hs.data(), st.p, sizeof(IsoState) * nqueries, cudaMemcpyDeviceToHost, s));
    int32_t herr = 0;
    NURI_CUDA(cudaMemcpyAsync(&herr, derr.p, 4, cudaMemcpyDeviceToHost, s));
    NURI_CUDA(cudaStreamSynchronize(s));
    if (herr & 4) NURI_FAIL(NURI_ERR_TIMEOUT, "nuri_topk_iso: time budget exhausted");
    {
      float ms = 0.f;
      NURI_CUDA(cudaEventElapsedTime(&ms, ev0, ev1));
      total.expand_ms += ms;
      total.expand_launches += 1;
    }
    total.expansions += hs[0].expansions;
    total.pruned += hs[0].pruned;
    total.dequeued += hs[0].dequeued;
    total.adj_bytes += hs[0].bytes;
    ++total.rounds;
    bool again = false;
    for (int i = 0; i < nqueries; ++i) {
      if (!active[i]) continue;
      final_state[i] = hs[i];
      if ((int64_t)hs[i].res_count > cap[i]) {
        again = true;
      }
    }
    if (!again) break;
    // overflowing queries run again with their final threshold and exact room; the others
    // keep nothing from this pass, so they are re-run too (their results were in `res`)
    ++restarts;
    for (int i = 0; i < nqueries; ++i) {
      if ((int64_t)hs[i].res_count > cap[i]) {
        tau_init[i] = hs[i].tau;
        // the histogram counted every result >= tau_final
        std::vector<int32_t> h(NBINS);
        NURI_CUDA(cudaMemcpyAsync(h.data(), hist.p + (int64_t)i * NBINS, sizeof(int32_t) * NBINS, cudaMemcpyDeviceToHost, s));
        NURI_CUDA(cudaStreamSynchronize(s));
        int64_t need = 0;
        for (int b = (int)(std::max<long long>(hs[i].tau, 0) >> prep[i].q.shift); b < NBINS; ++b) need += h[b];
        cap[i] = std::max<int64_t>(need + 64, cap[i]);
      } else {
        tau_init[i] = std::max<long long>(tau_init[i], hs[i].tau);
      }
    }
  }

  // ---- top-k merge over every query ----
  std::vector<long long> taus(nqueries);
  std::vector<int64_t> counts(nqueries);
  for (int i = 0; i < nqueries; ++i) {
    taus[i] = final_state[i].tau;
    counts[i] = std::min<int64_t>((int64_t)final_state[i].res_count, cap[i]);
  }
  int64_t maxsel = 0;
  for (int i = 0; i < nqueries; ++i) maxsel += counts[i];
  DBuf<long long> d_taus;
  DBuf<int64_t> d_counts;
  d_taus.alloc(nqueries, s);
  d_counts.alloc(nqueries, s);
  NURI_CUDA(cudaMemcpyAsync(d_taus.p, taus.data(), sizeof(long long) * nqueries, cudaMemcpyHostToDevice, s));
  NURI_CUDA(cudaMemcpyAsync(d_counts.p, counts.data(), sizeof(int64_t) * nqueries, cudaMemcpyHostToDevice, s));
  DBuf<int32_t> sel_q, sel_key, nsel;
  DBuf<long long> sel_score;
  sel_q.alloc(std::max<int64_t>(maxsel, 1), s);
  sel_score.alloc(std::max<int64_t>(maxsel, 1), s);
  sel_key.alloc(std::max<int64_t>(maxsel, 1) * KCOLS, s);
  nsel.alloc(1, s);
  NURI_CUDA(cudaMemsetAsync(nsel.p, 0, 4, s));
  if (maxsel > 0) {
    ++launches;
    k_iso_select<<<gridn(maxsel), 256, 0, s>>>(cx, nqueries, d_taus.p, d_counts.p, sel_q.p,
                                                sel_score.p, sel_key.p, nsel.p);
  }
  int32_t ns = 0;
  NURI_CUDA(cudaMemcpyAsync(&ns, nsel.p, 4, cudaMemcpyDeviceToHost, s));
  NURI_CUDA(cudaStreamSynchronize(s));
  int maxcols = 0;
  for (int i = 0; i < nqueries; ++i) maxcols = std::max(maxcols, QMAX + 2 * prep[i].q.ne);
  DBuf<int32_t> perm, perm2;
  perm.alloc(std::max(ns, 1), s);
  perm2.alloc(std::max(ns, 1), s);
  if (ns > 0) {
    ++launches;
    k_iota32<<<gridn(ns), 256, 0, s>>>(perm.p, ns);
    DBuf<uint32_t> k32, k32b;
    k32.alloc(ns, s);
    k32b.alloc(ns, s);
    size_t tb = 0;
    cub::DeviceRadixSort::SortPairs(nullptr, tb, k32.p, k32b.p, perm.p, perm2.p, ns, 0, 32, s);
    DBuf<unsigned long long> k64, k64b;
    k64.alloc(ns, s);
    k64b.alloc(ns, s);
    size_t tb2 = 0;
    cub::DeviceRadixSort::SortPairs(nullptr, tb2, k64.p, k64b.p, perm.p, perm2.p, ns, 0, 64, s);
    DBuf<uint8_t> tmp;
    tmp.alloc(std::max(tb, tb2), s);
    size_t tbx = std::max(tb, tb2);
    for (int col = maxcols - 1; col >= 0; --col) {
      if (col >= QMAX && ((col - QMAX) / 2) >= EMAX) continue;
      ++launches;
      k_iso_col<<<gridn(ns), 256, 0, s>>>(sel_key.p, perm.p, ns, col, k32.p);
      NURI_CUDA(cub::DeviceRadixSort::SortPairs(tmp.p, tbx, k32.p, k32b.p, perm.p, perm2.p, ns, 0, 32, s));
      std::swap(perm.p, perm2.p);
    }
    ++launches;
    k_iso_final_key<<<gridn(ns), 256, 0, s>>>(sel_q.p, sel_score.p, perm.p, ns, k64.p);
    NURI_CUDA(cub::DeviceRadixSort::SortPairs(tmp.p, tbx, k64.p, k64b.p, perm.p, perm2.p, ns, 0, 64, s));
    std::swap(perm.p, perm2.p);
  }
  // bring the sorted rows to the host (ns rows: query, score, key) and split per query
  std::vector<int32_t> h_perm(ns), h_q(std::max(ns, 1));
  std::vector<long long> h_score(std::max(ns, 1));
  std::vector<int32_t> h_key((size_t)std::max(ns, 1) * KCOLS);
  if (ns > 0) {
    NURI_CUDA(cudaMemcpyAsync(h_perm.data(), perm.p, sizeof(int32_t) * ns, cudaMemcpyDeviceToHost, s));
    NURI_CUDA(cudaMemcpyAsync(h_q.data(), sel_q.p, sizeof(int32_t) * ns, cudaMemcpyDeviceToHost, s));
    NURI_CUDA(cudaMemcpyAsync(h_score.data(), sel_score.p, sizeof(long long) * ns, cudaMemcpyDeviceToHost, s));
    NURI_CUDA(cudaMemcpyAsync(h_key.data(), sel_key.p, sizeof(int32_t) * ns * KCOLS, cudaMemcpyDeviceToHost, s));
    NURI_CUDA(cudaStreamSynchronize(s));
  }
  double ms = timer.stop();
  std::vector<std::vector<int32_t>> rows_of(nqueries);
  for (int i = 0; i < ns; ++i) {
    int32_t r = h_perm[i];
    rows_of[h_q[r]].push_back(r);
  }
  for (int qi = 0; qi < nqueries; ++qi) {
    const IsoQuery& Q = prep[qi].q;
    auto& rows = rows_of[qi];
    int32_t count = (int32_t)rows.size();
    if (!keep_ties) count = std::min<int32_t>(count, ks[qi]);
    nuri_result* r = new_result(1, count, (int64_t)count * Q.nq, (int64_t)count * Q.ne, false);
    for (int i = 0; i < count; ++i) {
      int32_t row = rows[i];
      r->score[i] = h_score[row];
      r->vert_off[i] = i * Q.nq;
      r->edge_off[i] = i * Q.ne;
      const int32_t* key = h_key.data() + (size_t)row * KCOLS;
      for (int a = 0; a < Q.nq; ++a) r->verts[i * Q.nq + a] = key[a];
      for (int e = 0; e < Q.ne; ++e) {
        r->edges[2 * (i * Q.ne + e)] = key[QMAX + 2 * e];
        r->edges[2 * (i * Q.ne + e) + 1] = key[QMAX + 2 * e + 1];
      }
    }
    r->vert_off[count] = count * Q.nq;
    r->edge_off[count] = count * Q.ne;
    nuri_stats st1 = total;
    st1.results_stored = (int64_t)final_state[qi].res_count;
    st1.threshold = final_state[qi].tau < 0 ? INT64_MIN : final_state[qi].tau;
    st1.restarts = restarts;
    st1.device_ms = ms;
    st1.launches = launches;
    r->stats = st1;
    outs[qi] = r;
  }
}

}  // namespace nuri
