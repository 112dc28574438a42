// Top-k cliques by size: Algorithm 1 (Section 3.2) with the clique user functions of
// Section 3.2 / Section 4.1 on the GPU.
//
//   P_s        = common neighbours of the members that come after every member in the
//                canonical order (Listing 1's set with the canonical extension of Section 3.2);
//                here the order is a degeneracy (core-peeling) rank (any total order enumerates
//                every clique exactly once; results are reported in original ids)
//   expandable = d in P_s;  relevant = true (all cliques) or maximality (flag)
//   bound      = |V_s| + |P_s| (Carraghan-Pardalos), tightened on adjacency bitmaps to
//                |V_s| + (colours of a greedy colouring of P_s); prune iff bound < tau (strict)
//   tau        = k-th best size among results found so far (global, atomicMax, monotone); in
//                the all-cliques ranking also lifted by subset counts (a c-clique holds
//                C(c, s) s-cliques) and by a greedy warm start before the search
//
// Work is organised as a bucketed best-first frontier driven from the host:
//   * seeds (one per vertex, Algorithm 1's initialisation) are sorted by bound and consumed in
//     descending-bound chunks (narrow seeds first); frontier records live in 1024 buckets
//     keyed by bound (LIFO inside a bucket, so the deepest records of the best bound go first);
//   * each round takes the highest bucket (or seed chunk) whose bound >= tau, topped up from
//     the next buckets when thin, and expands it with one warp per record (k_clique_expand);
//   * a record with |P| <= 64 is finished in place: the warp builds the 64x64 bit adjacency
//     of P in shared memory and its lanes search the record's subtrees (colour-ordered
//     branching over lane tasks);
//   * a record with 64 < |P| <= 512 goes to a dense tier (2, 4 or 8 words a row): its bitmap
//     is stored once and its search nodes become tasks of a global queue (k_clique_tasks),
//     coloured once each, with continuation tasks donated from busy lanes and tie-aware
//     pruning against the k-th tied result;
//   * a record with |P| > 512 is first coloured on a bitmap when |P| <= 1024 (dropped if the
//     colours cannot reach tau), else split: for every d in P the warp intersects the suffix
//     of P after d with N+(d) (binary search + ballot/popc), and children whose bound >= tau
//     go to a staging array that is scattered into the buckets;
//   * buckets that overflow the device frontier capacity are spilled to pinned host memory
//     (the role of the paper's disk-backed virtual priority queue, Section 5) and reloaded,
//     filtered by tau, when they become the highest bucket.
// Results (clique records with size >= tau when processed) are appended to a device buffer
// that is compacted in flight; a histogram of their sizes drives tau.  A final kernel sequence
// selects the rows with size >= tau, maps them to original ids, sorts them by (size desc, ids
// lex asc) and keeps k.
#include <cub/cub.cuh>

#include <algorithm>
#include <chrono>
#include <climits>
#include <condition_variable>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <thread>
#include <vector>

#include "nuri_internal.cuh"
#include "topk_common.cuh"

namespace nuri {
namespace {

constexpr int MAXD = 256;      // largest clique the records can hold
constexpr int NB = 1024;       // frontier buckets by bound (bucket NB-1 holds every bound
                               // >= NB-1; cliques never exceed MAXD < NB-1)
constexpr int PSMEM = 512;     // P entries staged in shared memory per warp
constexpr int CB_ROWS = 1024;  // candidates the split tier's colouring check handles
constexpr int CB_W = CB_ROWS / 64;

struct Rec {
  int32_t nv;
  int32_t bound;
  int32_t V[MAXD];  // ranks, ascending
};

struct QState {
  int32_t tau;
  int32_t err;           // bit 0: clique larger than MAXD; bit 2: time budget exhausted;
                         // bit 3: a corrupt frontier record (skipped, reported)
  int64_t res_count;     // results appended (may exceed the capacity: then a re-run)
  int64_t stage_count;   // children slots reserved in the staging array
  int64_t defer_count;   // parents sent back because the staging array was full
  int64_t wide_count;    // records handed to the 8-word bitmap tail
  int64_t mid_count;     // records handed to the 4-word bitmap tail
  int64_t small_count;   // records handed to the 2-word bitmap tail
  int64_t work_next;     // dynamic work counter
  unsigned long long expansions, pruned, dequeued, adj_bytes;
  unsigned long long tail_words;  // adjacency-row words combined by the task kernel
  unsigned long long lex_pruned;  // nodes pruned by the lexicographic tie bound
  int32_t hmax;          // largest clique size recorded so far
  int32_t bad_nv;        // err bit 3: a frontier record that is not a clique record ...
  int64_t bad_item;      // ... and its position in the launch's input
  int32_t hist[MAXD + 2];
};

// A query that runs under a time budget gets a watchdog thread: if the query is still running
// 20 s after its budget ran out (every kernel checks the deadline, so it should have ended),
// the thread reports on stderr, every 30 s, the source line of the query's last CUDA call and
// a snapshot of its device state (copied on a stream of its own), and never touches the query.
class QueryWatchdog {
 public:
  QueryWatchdog(const QState* dev_state, const std::atomic<int64_t>* rounds) {
    const uint64_t budget = time_budget_ns();
    if (!budget) return;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return;
    th_ = std::thread([this, dev_state, rounds, budget, dev] {
      using namespace std::chrono;
      const auto t0 = steady_clock::now();
      auto wait = nanoseconds(budget) + seconds(20);
      std::unique_lock<std::mutex> lk(mu_);
      while (!cv_.wait_for(lk, wait, [this] { return done_; })) {
        wait = seconds(30);
        // the host side first: no CUDA call, so that it is reported even when the query's
        // thread holds the driver
        fprintf(stderr,
                "[nuri] clique query still running %.0f s after its start: round %lld, last "
                "CUDA call at cliques/capi line %d\n",
                duration<double>(steady_clock::now() - t0).count(), (long long)rounds->load(),
                g_cuda_site.load(std::memory_order_relaxed));
        fflush(stderr);
        QState h;
        memset(&h, 0, sizeof(h));
        cudaSetDevice(dev);
        cudaStream_t ws = nullptr;
        bool copied = false;
        if (cudaStreamCreateWithFlags(&ws, cudaStreamNonBlocking) == cudaSuccess) {
          copied = cudaMemcpyAsync(&h, dev_state, sizeof(h), cudaMemcpyDeviceToHost, ws) ==
                       cudaSuccess &&
                   cudaStreamSynchronize(ws) == cudaSuccess;
          cudaStreamDestroy(ws);
        }
        fprintf(stderr,
                "[nuri]   device state%s: tau %d err %d results %lld work_next %lld staged "
                "%lld deferred %lld dense %lld/%lld/%lld nodes %llu\n",
                copied ? "" : " (not read)", h.tau, h.err, (long long)h.res_count,
                (long long)h.work_next,
                (long long)h.stage_count, (long long)h.defer_count, (long long)h.small_count,
                (long long)h.mid_count, (long long)h.wide_count, h.expansions);
        fflush(stderr);
      }
    });
  }
  ~QueryWatchdog() {
    if (!th_.joinable()) return;
    {
      std::lock_guard<std::mutex> lk(mu_);
      done_ = true;
    }
    cv_.notify_all();
    th_.join();
  }

 private:
  std::mutex mu_;
  std::condition_variable cv_;
  bool done_ = false;
  std::thread th_;
};

__device__ __forceinline__ int lower_bound_dev(const int32_t* a, int lo, int hi, int32_t x) {
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    if (a[mid] < x) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

__device__ __forceinline__ int64_t lower_bound_dev64(const int32_t* a, int64_t lo, int64_t hi,
                                                     int32_t x) {
  while (lo < hi) {
    int64_t mid = (lo + hi) >> 1;
    if (__ldg(a + mid) < x) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

__device__ __forceinline__ bool contains64(const int32_t* a, int64_t lo, int64_t hi, int32_t x) {
  int64_t p = lower_bound_dev64(a, lo, hi, x);
  return p < hi && __ldg(a + p) == x;
}

// Is the clique C (ranks) maximal, i.e. does no vertex outside it touch every member?
__device__ bool is_maximal(const DevGraph& g, const int32_t* C, int c) {
  int best = 0;
  int32_t bestdeg = INT32_MAX;
  int32_t ids[MAXD + 1];
  for (int i = 0; i < c; ++i) {
    ids[i] = __ldg(g.vert_of + C[i]);
    int32_t d = __ldg(g.deg + ids[i]);
    if (d < bestdeg) {
      bestdeg = d;
      best = i;
    }
  }
  int64_t b = g.off[ids[best]], e = g.off[ids[best] + 1];
  for (int64_t t = b; t < e; ++t) {
    int32_t w = __ldg(g.adj + t);
    bool all = true;
    for (int i = 0; i < c && all; ++i) {
      if (i == best) continue;
      if (ids[i] == w) {
        all = false;
        break;
      }
      all = contains64(g.adj, g.off[ids[i]], g.off[ids[i] + 1], w);
    }
    if (all) return false;
  }
  return true;
}

struct Ctx {
  DevGraph g;
  QState* st;
  Rec* res;
  int64_t res_cap;
  Rec* stage;
  int64_t stage_cap;
  Rec* deferred;
  Rec* wide;            // records for the 8-word bitmap tail (256 < |P| <= 512)
  Rec* mid;             // records for the 4-word bitmap tail (128 < |P| <= 256)
  Rec* small;           // records for the 2-word bitmap tail (64 < |P| <= 128)
  int32_t* pscratch;    // per-warp global P buffer (max_out entries each)
  unsigned long long* cbits;  // per-warp adjacency bitmap (CB_ROWS x CB_W words) for the
                              // colouring check of split records; null when unused
  int64_t pscratch_stride;
  int32_t k;
  int32_t maximal;
  int32_t no_prune;
  const uint64_t* deadline;  // global timer value after which the query stops (err bit 2)
  int32_t split_above;       // records with more candidates than this are split
};

__device__ __forceinline__ bool past_deadline(const Ctx& cx) {
  return global_ns() > *(const volatile uint64_t*)cx.deadline;
}

// Largest s with C(c, s) >= k (0 when there is none): a clique of size c holds that many
// cliques of size s, so the k-th best clique size is at least s.
__device__ __forceinline__ int subset_tau(int c, int k) {
  double b = 1.0;  // C(c, s)
  int s = c;
  while (s > 1 && b < (double)k) {
    b = b * s / (double)(c - s + 1);
    --s;
  }
  return b >= (double)k ? s : 0;
}

// Append one clique (ranks) of size c as a candidate result and refresh tau.
__device__ void add_result(const Ctx& cx, const int32_t* V, int nv, int32_t extra_count,
                           const int32_t* extra) {
  int c = nv + extra_count;
  int64_t slot = (int64_t)atomicAdd((unsigned long long*)&cx.st->res_count, 1ull);
  if (slot < cx.res_cap) {
    Rec* r = cx.res + slot;
    r->nv = c;
    r->bound = c;
    for (int i = 0; i < nv; ++i) r->V[i] = V[i];
    for (int i = 0; i < extra_count; ++i) r->V[nv + i] = extra[i];
  }
  atomicAdd(&cx.st->hist[c], 1);
  if (c > ld_volatile(&cx.st->hmax)) atomicMax(&cx.st->hmax, c);
  if (!cx.maximal && c > ld_volatile(&cx.st->tau)) {
    // every subset of a clique is a clique: one of size c holds C(c, s) cliques of size s, so
    // the k-th best size is at least the largest such s with C(c, s) >= k
    const int s = subset_tau(c, cx.k);
    if (s > ld_volatile(&cx.st->tau)) atomicMax(&cx.st->tau, s);
  }
  if ((int64_t)(slot + 1) < (int64_t)cx.k) return;  // fewer than k results so far
  publish_threshold(cx.st->hist, ld_volatile(&cx.st->hmax), 0, cx.k, &cx.st->tau);
}

// ---------------------------------------------------------------------------------------------
// Expansion kernel: one warp per record (dynamic assignment).
//   seeds != nullptr: record i is the seed vertex seeds[i] (nv = 1)
//   otherwise       : record i is in[i]
// W = 64-bit words of the bitmap tail: records with |P| <= 64 W are finished in the warp.
// The W = 1 instantiation hands records with 64 < |P| <= 64 KWIDE to the wide instantiation
// (cx.wide list) and splits records with larger |P|; the wide one splits only the latter.
// ---------------------------------------------------------------------------------------------
constexpr int KWIDE = 8;

template <int W>
struct KCfg {
  static constexpr int WARPS = 4;
};
template <>
struct KCfg<KWIDE> {
  static constexpr int WARPS = 2;
};

template <int W>
__device__ __forceinline__ int lowest(const unsigned long long* X, int wa) {
#pragma unroll
  for (int q = 0; q < W; ++q)
    if (q < wa && X[q]) return q * 64 + __ffsll((long long)X[q]) - 1;
  return -1;
}

template <int W>
__device__ __forceinline__ int highest(const unsigned long long* X, int wa) {
#pragma unroll
  for (int q = W - 1; q >= 0; --q)
    if (q < wa && X[q]) return q * 64 + 63 - __clzll((long long)X[q]);
  return -1;
}

template <int W>
__device__ __forceinline__ int popc(const unsigned long long* X, int wa) {
  int c = 0;
#pragma unroll
  for (int q = 0; q < W; ++q)
    if (q < wa) c += __popcll(X[q]);
  return c;
}

template <int W>
__device__ __forceinline__ bool any(const unsigned long long* X, int wa) {
  unsigned long long a = 0;
#pragma unroll
  for (int q = 0; q < W; ++q)
    if (q < wa) a |= X[q];
  return a != 0;
}

// single-bit updates through unrolled predicated loops: the masks stay in registers
// (an index computed at run time would move the whole array to local memory)
template <int W>
__device__ __forceinline__ void clear_bit(unsigned long long* X, int v) {
#pragma unroll
  for (int q = 0; q < W; ++q)
    if (q == (v >> 6)) X[q] &= ~(1ull << (v & 63));
}

template <int W>
__device__ __forceinline__ void set_bit(unsigned long long* X, int v) {
#pragma unroll
  for (int q = 0; q < W; ++q)
    if (q == (v >> 6)) X[q] |= 1ull << (v & 63);
}

// X &= ~row over the words of X that can be non-zero: from q0 (X is zero below word q0) up to
// wa (the candidate count's words).  A store row is 16-byte aligned (W >= 2), so it is read
// two words per load and only the pairs that overlap [q0, wa) are read.
template <int W>
__device__ __forceinline__ void andnot_live(unsigned long long* X, const unsigned long long* row,
                                            int q0, int wa) {
  static_assert(W % 2 == 0, "paired row loads need an even word count");
#pragma unroll
  for (int q = 0; q < W; q += 2)
    if (q + 1 >= q0 && q < wa) {
      const ulonglong2 r = *reinterpret_cast<const ulonglong2*>(row + q);
      X[q] &= ~r.x;
      X[q + 1] &= ~r.y;
    }
}

// One greedy colour class: the members of cls, taken in index order, that have no neighbour
// among the members taken before them; each member also leaves R.  The class is built word
// by word (unrolled, so every mask index is a compile-time constant): when word q is reached,
// the words below it are already empty, so a member's row is applied from its own word pair
// on.  cls is empty on return.
template <int W>
__device__ __forceinline__ void colour_class(unsigned long long* cls, unsigned long long* R,
                                             const unsigned long long* rows, int wa,
                                             unsigned long long& my_words) {
  static_assert(W % 2 == 0, "paired row loads need an even word count");
#pragma unroll
  for (int q = 0; q < W; ++q) {
    if (q < wa) {
      while (cls[q]) {
        const int b = __ffsll((long long)cls[q]) - 1;
        const unsigned long long bit = 1ull << b;
        cls[q] &= ~bit;
        R[q] &= ~bit;
        const unsigned long long* row = rows + (int64_t)(q * 64 + b) * W;
#pragma unroll
        for (int r = q & ~1; r < W; r += 2)
          if (r < wa) {
            const ulonglong2 x = *reinterpret_cast<const ulonglong2*>(row + r);
            cls[r] &= ~x.x;
            cls[r + 1] &= ~x.y;
          }
        my_words += wa - q;
      }
    }
  }
}

// Core filter of a record's candidates (warp-cooperative): rows[i*W .. i*W+W) is the adjacency
// of candidate i among the p candidates.  Candidates with fewer than need - 1 neighbours among
// the kept ones are dropped, repeatedly, until every kept candidate has enough (the (need-1)-
// core of P); a dropped candidate's row is cleared and its bit removed from every row.
// Returns the number kept.  alive: W words of shared memory.
template <int W>
__device__ int core_peel(unsigned long long* rows, int p, int need, unsigned long long* alive,
                         int lane) {
  const unsigned FULL = 0xffffffffu;
  if (lane < W) {
    const int lo = lane * 64;
    alive[lane] = p >= lo + 64 ? ~0ull : (p > lo ? (1ull << (p - lo)) - 1 : 0ull);
  }
  __syncwarp();
  bool any_removed = false;
  while (true) {
    bool removed = false;
    for (int i = lane; i < p; i += 32) {
      if (!((alive[i >> 6] >> (i & 63)) & 1ull)) continue;
      int d = 0;
#pragma unroll
      for (int q = 0; q < W; ++q) d += __popcll(rows[i * W + q] & alive[q]);
      if (d < need - 1) {
        atomicAnd(&alive[i >> 6], ~(1ull << (i & 63)));
        removed = true;
      }
    }
    __syncwarp();
    if (!__any_sync(FULL, removed)) break;
    any_removed = true;
  }
  if (any_removed) {
    for (int i = lane; i < p; i += 32) {
      const bool a = (alive[i >> 6] >> (i & 63)) & 1ull;
#pragma unroll
      for (int q = 0; q < W; ++q) rows[i * W + q] = a ? (rows[i * W + q] & alive[q]) : 0ull;
    }
  }
  int c = 0;
#pragma unroll
  for (int q = 0; q < W; ++q) c += __popcll(alive[q]);
  __syncwarp();
  return c;
}

// out = a & row over words [0, wa) (the words at and above wa are zero in a), paired loads.
template <int W>
__device__ __forceinline__ void and_live(unsigned long long* out, const unsigned long long* a,
                                         const unsigned long long* row, int wa) {
  static_assert(W % 2 == 0, "paired row loads need an even word count");
#pragma unroll
  for (int q = 0; q < W; q += 2)
    if (q < wa) {
      const ulonglong2 r = *reinterpret_cast<const ulonglong2*>(row + q);
      out[q] = a[q] & r.x;
      out[q + 1] = a[q + 1] & r.y;
    } else {
      out[q] = 0ull;
      out[q + 1] = 0ull;
    }
}

// ---------------------------------------------------------------------------------------------
// Dense records (64 < |P| <= 512) are searched through a global task queue.  The warp that
// dequeues such a record builds its adjacency bitmap once and stores it, with the vertex of
// every candidate index and the record's vertices, in a store slot (global memory; a few MB,
// L2-resident).  Every search node whose candidate set is still large becomes a task that any
// lane of the GPU can take; nodes with at most `split_bits` candidates are finished by the
// lane that takes them.  Tasks are processed in waves until none is left.  Once a wave's input
// is used up, a lane still inside a subtree hands the rest of its search stack on as
// continuation tasks (nodes already visited, with the candidates not yet branched on), so the
// next wave spreads that subtree over the GPU instead of leaving it to one lane.
// ---------------------------------------------------------------------------------------------
constexpr int kSliceNodes = 1 << 14;  // nodes a lane searches before it sheds work
constexpr int kShed = 8;              // levels shed at a time
constexpr int kFullHandOff = 64;      // pending levels a lane hands on in one go
constexpr int kTieDefer = 8;          // vertices a tie node must need to be put back
constexpr int64_t kTieQueue = 1 << 18;  // tie nodes put back at most (per chunk of records)
// Device memory bounds of one query's buffers (they make the server's admission estimate an
// upper bound): records handed to the dense tiers or sent back per round, and the dense store
constexpr int64_t kRoundRecs = 1 << 16;
constexpr int64_t kDefaultFrontier = 1 << 20;  // device frontier records before spilling
constexpr int64_t kStoreBytes = 256ll << 20;

struct WTask {
  int32_t slot;
  int16_t depth;  // depth + 1 candidates are picked below the record
  int16_t cont;   // 1: the node was visited already; only its branching remains;
                  // 2: as 1, a tie node put back once (searched when taken)
  unsigned long long C[KWIDE];            // the picked candidates (a set: any depth)
  unsigned long long P[KWIDE], X[KWIDE];  // X only in maximal mode
};

// The picked candidates pick[0..d] of a node as a task's set.
__device__ __forceinline__ void write_picks(WTask* t, const uint16_t* pick, int d) {
  unsigned long long c[KWIDE];
#pragma unroll
  for (int q = 0; q < KWIDE; ++q) c[q] = 0ull;
  for (int q = 0; q <= d; ++q) set_bit<KWIDE>(c, pick[q]);
#pragma unroll
  for (int q = 0; q < KWIDE; ++q) t->C[q] = c[q];
}

struct WideStore {
  unsigned long long* rows;  // per slot: BMW * W words (row i = words i*W .. i*W+W)
  int32_t* vmap;             // per slot: BMW vertex ranks
  int32_t* recV;             // per slot: MAXD record vertices
  int32_t* recN;             // per slot: record size
  int32_t* recP;             // per slot: number of candidates
  unsigned long long* nslots;
  int64_t slot_cap;
  WTask* q_out;
  unsigned long long* q_count;
  int64_t q_cap;
  int32_t split_bits;
  const unsigned long long* in_next;  // fetch counter of the wave's input (tasks kernel)
  int64_t in_n;                       // tasks in the wave's input
  // tie-aware pruning (all-cliques ranking): at least k known results rank before every
  // clique of size lex_tau whose smallest vertex id exceeds lex_first.  low (per slot, W
  // words) marks the candidates with id <= lex_first, reclow the slots whose record holds
  // such a vertex.  lex_tau = INT32_MIN: off.
  const unsigned long long* low;
  const int32_t* reclow;
  int32_t lex_tau;
  int32_t lex_first;
  // full lexicographic bound: per slot the original id of every candidate (cid), the
  // candidates in ascending id order (byid) and the record's ids ascending (rid); lexL: the
  // sorted id list of the (k - c_hi)-th smallest stored result of size lex_tau (null: off)
  int32_t* cid;
  uint16_t* byid;
  int32_t* rid;
  const int32_t* lexL;
  // tie nodes put back until the task queue runs dry (null: searched where met)
  WTask* q_tie;
  unsigned long long* tie_count;
  int64_t tie_cap;
};

// Does every clique of size tau below the node rank after the list lexL?  The node's
// smallest possible sorted id list merges the record's ids (rid), the picked candidates and
// the m smallest candidates of Pn (walking the candidates in id order); it is compared with
// lexL element by element.  True only when it is larger (equal or smaller: keep the node).
template <int W>
__device__ bool lex_list_after(const WideStore& ws, int slot, int nv, const uint16_t* pick,
                               int depth, const unsigned long long* Pn, int m, int tau) {
  constexpr int BMW = 64 * W;
  const int32_t* rid = ws.rid + (int64_t)slot * MAXD;
  const int32_t* cid = ws.cid + (int64_t)slot * BMW;
  const uint16_t* byid = ws.byid + (int64_t)slot * BMW;
  const int p = ws.recP[slot];
  unsigned long long picked[W];
#pragma unroll
  for (int q = 0; q < W; ++q) picked[q] = 0ull;
  for (int q = 0; q <= depth; ++q) set_bit<W>(picked, pick[q]);
  int ir = 0, ic = 0, taken = 0;
  int32_t cand = INT32_MAX;  // id of the next candidate stream element
  auto next_cand = [&]() {
    cand = INT32_MAX;
    while (ic < p) {
      const int a = byid[ic++];
      const int qa = a >> 6;
      unsigned long long pw = 0, pp = 0;
#pragma unroll
      for (int q = 0; q < W; ++q)
        if (q == qa) {
          pw = picked[q];
          pp = Pn[q];
        }
      const unsigned long long bit = 1ull << (a & 63);
      if (pw & bit) {
        cand = cid[a];
        return;
      }
      if ((pp & bit) && taken < m) {
        ++taken;
        cand = cid[a];
        return;
      }
    }
  };
  next_cand();
  for (int t = 0; t < tau; ++t) {
    int32_t x;
    if (ir < nv && rid[ir] < cand) x = rid[ir++];
    else {
      x = cand;
      next_cand();
    }
    const int32_t y = ws.lexL[t];
    if (x != y) return x > y;
  }
  return false;
}

// Search below a tie node: no clique below the node exceeds T = tau (its colour bound equals
// T), so the cliques of size T that can still rank in the top k are the smallest ones by
// sorted id list.  Adding one vertex set S to the fixed clique of the node keeps the order of
// the S parts, so S is built in ascending id order: level l (l vertices chosen) tries its
// candidates by increasing id, the child of candidate c keeps the untried candidates (all of
// larger id) adjacent to c, and a level ends once a colouring shows that its untried
// candidates cannot complete a clique of size T.  Cliques come out in increasing order; after
// k of them every later clique here has k results before it, and the search stops (all-cliques
// ranking, ties cut at k).  Levels use lev[0 .. need), cursor positions cur[0 .. need).
template <int W>
__device__ void tie_search(const Ctx& cx, const WideStore& ws, int slot, int depth,
                           uint16_t* pick, const unsigned long long* P0, int T,
                           unsigned long long (*lev)[W], uint16_t* cur, int32_t& t_cache,
                           unsigned long long& my_exp, unsigned long long& my_words,
                           unsigned long long& my_lex, bool& out_of_time) {
  constexpr int BMW = 64 * W;
  const unsigned long long* rows = ws.rows + (int64_t)slot * BMW * W;
  const int32_t* vmap = ws.vmap + (int64_t)slot * BMW;
  const int32_t* recV = ws.recV + (int64_t)slot * MAXD;
  const uint16_t* byid = ws.byid + (int64_t)slot * BMW;
  const int nv = ws.recN[slot];
  const int p = ws.recP[slot];
  const int wa = (p + 63) >> 6;
  const int need = T - (nv + depth + 1);
  int emitted = 0;
#pragma unroll
  for (int q = 0; q < W; ++q) lev[0][q] = q < wa ? P0[q] : 0ull;
  cur[0] = 0;
  int l = 0;
  while (l >= 0) {
    ++my_exp;
    if ((my_exp & 31) == 0) {
      t_cache = ld_volatile(&cx.st->tau);
      if ((my_exp & 1023) == 0 && past_deadline(cx)) {
        atomicOr(&cx.st->err, 4);
        out_of_time = true;
      }
    }
    if (out_of_time || t_cache > T) return;  // every clique left here is below the threshold
    // the level's bound: its untried candidates must hold need - l more colours
    unsigned long long R[W];
#pragma unroll
    for (int q = 0; q < W; ++q) R[q] = lev[l][q];
    for (int c = 1; c < need - l && any<W>(R, wa); ++c) {
      unsigned long long cls[W];
#pragma unroll
      for (int q = 0; q < W; ++q) cls[q] = R[q];
      colour_class<W>(cls, R, rows, wa, my_words);
    }
    if (!any<W>(R, wa)) {
      --l;
      continue;
    }
    // the untried candidate of smallest id
    int c = -1;
    while (cur[l] < p) {
      const int a = byid[cur[l]++];
      unsigned long long w = 0;
#pragma unroll
      for (int q = 0; q < W; ++q)
        if (q == (a >> 6)) w = lev[l][q];
      if ((w >> (a & 63)) & 1ull) {
        c = a;
        break;
      }
    }
    if (c < 0) {
      --l;
      continue;
    }
    clear_bit<W>(lev[l], c);
    pick[depth + 1 + l] = (uint16_t)c;
    if (l + 1 == need) {  // a clique of size T
      int32_t pr[MAXD];
      for (int q = 0; q <= depth + 1 + l; ++q) pr[q] = vmap[pick[q]];
      add_result(cx, recV, nv, depth + 2 + l, pr);
      if (++emitted >= cx.k) {
        ++my_lex;  // the rest of the subtree ranks after these k
        return;
      }
      continue;
    }
    and_live<W>(lev[l + 1], lev[l], rows + c * W, wa);
    my_words += wa;
    cur[l + 1] = cur[l];  // the child's candidates all have larger ids
    ++l;
  }
}

// Visit the node (record + picks[0..depth], candidates Pn, explored Xn) of a dense record and
// finish its subtree with colour-ordered branching; if `split` is set and the node has more
// than split_bits candidates, its viable children become tasks instead (colour order: child
// s_t has the candidates before it adjacent to it, the explored set plus the candidates after
// it, and the bound |node| + colour(s_t)).
template <int W>
__device__ void dense_node(const Ctx& cx, const WideStore& ws, int slot, int depth,
                           uint16_t* pick, unsigned long long* Pn, unsigned long long* Xn,
                           bool split, int cont, int32_t& t_cache, unsigned long long& my_exp,
                           unsigned long long& my_pruned, unsigned long long& my_words,
                           unsigned long long& my_lex, bool& limit_hit, bool& out_of_time) {
  constexpr int BMW = 64 * W;
  const unsigned long long* rows = ws.rows + (int64_t)slot * BMW * W;
  const int32_t* vmap = ws.vmap + (int64_t)slot * BMW;
  const int32_t* recV = ws.recV + (int64_t)slot * MAXD;
  const int nv = ws.recN[slot];
  const int p = ws.recP[slot];
  const int wa = (p + 63) >> 6;
  const DevGraph& g = cx.g;
  // Level l keeps rem (candidates not yet branched on), R (high-colour candidates not yet
  // branched on) and, in maximal mode, X (explored); a tie search below level l uses the levels
  // above it.
  unsigned long long stkP[MAXD][W];
  unsigned long long stkR[MAXD][W];
  unsigned long long stkX[MAXD][W];
  uint16_t tcur[MAXD];
  const int base_depth = depth;

  // Tie nodes (colour bound equal to tau) of a near-complete candidate set (the clique must
  // take at least half of the candidates) are searched in id order (tie_search).  One that
  // needs kTieDefer or more vertices is first put back as a task (cont = 2) in the tie queue,
  // which runs once the task queue is empty: by then the other searches may have raised tau
  // past it, and it is dropped unsearched.  A task put back once, or a node that finds no room
  // in the tie queue, is searched at once.
  const bool tie_ok = ws.cid != nullptr && !cx.maximal && !cx.no_prune;
  auto tie_node = [&](int d, const unsigned long long* P_, int size) -> bool {
    const int need = t_cache - size;
    if (!tie_ok || t_cache == INT32_MIN || t_cache > MAXD || need < 1 || d + need >= MAXD ||
        2 * need < popc<W>(P_, wa))
      return false;
    // the node's smallest possible sorted id list ranks after the (k - c_hi)-th known result
    // of size tau: so does every clique below it
    if (ws.lexL && ws.lex_tau == t_cache &&
        lex_list_after<W>(ws, slot, nv, pick, d, P_, need, t_cache)) {
      ++my_pruned;
      ++my_lex;
      return true;
    }
    if (split && ws.q_tie && !(cont == 2 && d == base_depth) && need >= kTieDefer &&
        (int64_t)ld_volatile(ws.tie_count) < ws.tie_cap) {
      const unsigned long long b = atomicAdd(ws.tie_count, 1ull);
      if ((int64_t)b < ws.tie_cap) {
        WTask* t = ws.q_tie + b;
        t->slot = slot;
        t->depth = (int16_t)d;
        t->cont = 2;
        write_picks(t, pick, d);
#pragma unroll
        for (int q = 0; q < KWIDE; ++q) t->P[q] = q < wa ? P_[q] : 0ull;
        return true;
      }
    }
    tie_search<W>(cx, ws, slot, d, pick, P_, t_cache, stkR + d + 1, tcur + d + 1, t_cache,
                  my_exp, my_words, my_lex, out_of_time);
    return true;
  };

  auto visit_node = [&](int d, const unsigned long long* P_, const unsigned long long* X_) {
    int size = nv + d + 1;
    ++my_exp;
    if ((my_exp & 31) == 0) {
      t_cache = ld_volatile(&cx.st->tau);
      if ((my_exp & 1023) == 0 && past_deadline(cx)) {
        atomicOr(&cx.st->err, 4);
        out_of_time = true;
      }
    }
    if (size >= t_cache) {
      bool rel = true;
      if (cx.maximal) {
        if (any<W>(P_, wa) || any<W>(X_, wa)) rel = false;
        else {
          int32_t C[MAXD];
          for (int a = 0; a < nv; ++a) C[a] = recV[a];
          for (int q = 0; q <= d; ++q) C[nv + q] = vmap[pick[q]];
          rel = is_maximal(g, C, size);
        }
      }
      if (rel) {
        int32_t pr[MAXD];
        for (int q = 0; q <= d; ++q) pr[q] = vmap[pick[q]];
        add_result(cx, recV, nv, d + 1, pr);
        t_cache = ld_volatile(&cx.st->tau);
      }
    }
  };

  if (!cont) visit_node(depth, Pn, Xn);
  if (out_of_time || !any<W>(Pn, wa)) return;
  if (nv + depth + 1 >= MAXD) {
    limit_hit = true;
    return;
  }
  if (split && depth + 2 < MAXD && popc<W>(Pn, wa) > ws.split_bits &&
      (int64_t)ld_volatile(ws.q_count) < ws.q_cap / 8) {
    // children as tasks, in colour order: count the viable ones, reserve their queue slots,
    // then emit them
    const int size = nv + depth + 1;
    const int cmin = (cx.no_prune || t_cache == INT32_MIN) ? 0 : t_cache - size;
    auto walk = [&](auto&& f) {
      unsigned long long left[W], prefix[W];
#pragma unroll
      for (int q = 0; q < W; ++q) {
        left[q] = Pn[q];
        prefix[q] = 0;
      }
      int c = 0;
      while (any<W>(left, wa)) {
        ++c;
        unsigned long long cls[W];
#pragma unroll
        for (int q = 0; q < W; ++q) cls[q] = left[q];
        int v;
        while ((v = lowest<W>(cls, wa)) >= 0) {
          andnot_live<W>(cls, rows + v * W, v >> 6, wa);
          my_words += wa - (v >> 6);
          clear_bit<W>(cls, v);
          clear_bit<W>(left, v);
          f(v, c, prefix);
          set_bit<W>(prefix, v);
        }
      }
    };
    int r = 0, colours = 0;
    walk([&](int, int c, const unsigned long long*) {
      if (c >= cmin) ++r;
      colours = c;
    });
    if (r > 0 && size + colours == t_cache && tie_node(depth, Pn, size)) return;
    my_pruned += (unsigned long long)(popc<W>(Pn, wa) - r);
    if (r == 0) return;
    const unsigned long long base = atomicAdd(ws.q_count, (unsigned long long)r);
    if ((int64_t)(base + r) <= ws.q_cap) {
      int k = 0;
      walk([&](int v, int c, const unsigned long long* prefix) {
        if (c < cmin) return;
        WTask* t = ws.q_out + base + (k++);
        my_words += wa;
        t->slot = slot;
        t->depth = (int16_t)(depth + 1);
        pick[depth + 1] = (uint16_t)v;
        write_picks(t, pick, depth + 1);
#pragma unroll
        for (int q = 0; q < KWIDE; ++q) {
          unsigned long long rq = q < W ? rows[v * W + q] : 0ull;
          unsigned long long pq = q < W ? Pn[q] : 0ull, xq = q < W ? Xn[q] : 0ull;
          unsigned long long pre = q < W ? prefix[q] : 0ull;
          t->P[q] = pre & rq;
          // explored: X, and the candidates after v in the colour order
          if (cx.maximal) t->X[q] = (xq | (pq & ~pre)) & rq;
        }
        t->cont = 0;
      });
      return;
    }
    // no room: mark the reserved slots that exist as empty and explore here
    for (unsigned long long q = base; q < base + r && (int64_t)q < ws.q_cap; ++q)
      ws.q_out[q].slot = -1;
  }
  // ---- finish the subtree here: colour once per node, branch over its high-colour set ----
  // A node's R is what is left of its candidates after greedy colour classes
  // 1 .. tau - |node| - 1 (those that cannot lift a clique to tau) are taken out; its children
  // come from R, highest index first, child u having the candidates (rem - u) & N(u), so each
  // clique below the node is reached once, through the first of its vertices to be branched
  // on.  The colouring is done once per node.
  int local = 0;      // nodes entered by this call
  bool fresh = true;  // the node at `depth` (candidates Pn) has not been coloured yet
  // lowc[d]: the clique at depth d holds a vertex with id <= lex_first (tie-aware pruning)
  const bool lex = ws.lex_tau != INT32_MIN;
  const unsigned long long* lowm = lex ? ws.low + (int64_t)slot * W : nullptr;
  uint8_t lowc[MAXD + 1];
  if (lex) {
    bool lc = ws.reclow[slot] != 0;
    for (int q = 0; q <= depth && !lc; ++q) lc = (lowm[pick[q] >> 6] >> (pick[q] & 63)) & 1ull;
    lowc[depth] = lc ? 1 : 0;
  }
  while (!out_of_time) {
    bool level_ok = true;
    if (fresh) {
      fresh = false;
      const int size = nv + depth + 1;
      // past kSliceNodes nodes while the wave still has input, every 1024 nodes: shed the
      // untried branches of the (at most kShed) shallowest levels below the current node as
      // tasks and keep searching the current path, so that deep searches spread over the
      // next waves (between which the host refreshes the threshold and the tie bound).  A
      // shed level's remaining cliques are those inside its untried candidates: the task
      // (cont = 1, candidates = the untried set) enumerates them; the level here stops.
      const bool drained = (int64_t)ld_volatile(ws.in_next) >= ws.in_n;
      if (split && local >= (drained ? 1024 : kSliceNodes) && (local & 1023) == 0 &&
          (int64_t)ld_volatile(ws.q_count) < ws.q_cap / 2) {
        int r = 0;
        for (int l = base_depth; l < depth && r < kShed; ++l) r += any<W>(stkR[l], wa) ? 1 : 0;
        if (r > 0) {
          const unsigned long long base = atomicAdd(ws.q_count, (unsigned long long)r);
          if ((int64_t)(base + r) <= ws.q_cap) {
            int k = 0;
            for (int l = base_depth; l < depth && k < r; ++l) {
              if (!any<W>(stkR[l], wa)) continue;
              WTask* t = ws.q_out + base + (k++);
              t->slot = slot;
              t->depth = (int16_t)l;
              t->cont = 1;
              write_picks(t, pick, l);
#pragma unroll
              for (int q = 0; q < KWIDE; ++q) {
                t->P[q] = q < wa ? stkP[l][q] : 0ull;
                if (cx.maximal) t->X[q] = q < wa ? stkX[l][q] : 0ull;
              }
#pragma unroll
              for (int q = 0; q < W; ++q)
                if (q < wa) stkR[l][q] = 0ull;
            }
          } else {
            for (unsigned long long q = base; q < base + r && (int64_t)q < ws.q_cap; ++q)
              ws.q_out[q].slot = -1;
          }
        }
      }
      // hand the rest of the stack on once the wave's input is used up (and there is room):
      // the current node and every level below it that still has vertices to branch on.  A
      // stack with more than kFullHandOff such levels, or a hand-off that found no room, is
      // shed a few levels at a time instead (above).
      if (split && ++local >= 16 && (local & 15) == 0 && drained &&
          (int64_t)ld_volatile(ws.q_count) < ws.q_cap / 2) {
        int r = any<W>(Pn, wa) ? 1 : 0;
        for (int l = base_depth; l < depth; ++l) r += any<W>(stkR[l], wa) ? 1 : 0;
        if (r == 0) break;
        const unsigned long long base =
            r <= kFullHandOff ? atomicAdd(ws.q_count, (unsigned long long)r) : ~0ull;
        if (r <= kFullHandOff && (int64_t)(base + r) <= ws.q_cap) {
          int k = 0;
          for (int l = base_depth; l <= depth; ++l) {
            if (l < depth ? !any<W>(stkR[l], wa) : !any<W>(Pn, wa)) continue;
            const unsigned long long* PL = l < depth ? stkP[l] : Pn;
            const unsigned long long* XL = l < depth ? stkX[l] : Xn;
            WTask* t = ws.q_out + base + (k++);
            t->slot = slot;
            t->depth = (int16_t)l;
            t->cont = 1;
            write_picks(t, pick, l);
#pragma unroll
            for (int q = 0; q < KWIDE; ++q) {
              t->P[q] = q < wa ? PL[q] : 0ull;
              if (cx.maximal) t->X[q] = q < wa ? XL[q] : 0ull;
            }
          }
          return;
        }
        if (r <= kFullHandOff)
          for (unsigned long long q = base; q < base + r && (int64_t)q < ws.q_cap; ++q)
            ws.q_out[q].slot = -1;
      }
      unsigned long long R[W];
#pragma unroll
      for (int q = 0; q < W; ++q) R[q] = Pn[q];
      level_ok = any<W>(R, wa);
      if (level_ok && size >= MAXD) {
        limit_hit = true;
        level_ok = false;
      }
      if (level_ok && !cx.no_prune && size + popc<W>(R, wa) < t_cache) {  // |V| + |P| < tau
        ++my_pruned;
        level_ok = false;
      }
      if (level_ok && !cx.no_prune && size < t_cache) {
        const int kmin = t_cache - size;  // classes 1 .. kmin-1 cannot reach tau
        for (int c = 1; c < kmin && any<W>(R, wa); ++c) {
          unsigned long long cls[W];
#pragma unroll
          for (int q = 0; q < W; ++q) cls[q] = R[q];
          colour_class<W>(cls, R, rows, wa, my_words);
        }
        if (!any<W>(R, wa)) {
          ++my_pruned;
          level_ok = false;
        }
      }
      // tie-aware pruning: when no clique below this node can exceed tau (one more colour
      // class empties R), every clique below it has size at most tau, and its sorted id list
      // is at least the node's smallest possible one: the clique's ids with the tau - |node|
      // smallest ids among the candidates.  If that list ranks after the (k - c_hi)-th stored
      // result of size tau, at least k known results rank before each of them.  The cheap
      // first test: neither the clique nor a candidate holds an id up to that result's first.
      if (level_ok && lex && ws.lex_tau == t_cache && size < t_cache) {
        unsigned long long hit = 0;
#pragma unroll
        for (int q = 0; q < W; ++q)
          if (q < wa) hit |= Pn[q] & lowm[q];
        const bool first_after = !hit && !lowc[depth];
        if (first_after || ws.lexL) {
          unsigned long long cls[W], R2[W];
#pragma unroll
          for (int q = 0; q < W; ++q) {
            cls[q] = R[q];
            R2[q] = R[q];
          }
          colour_class<W>(cls, R2, rows, wa, my_words);
          if (!any<W>(R2, wa) &&
              (first_after ||
               lex_list_after<W>(ws, slot, nv, pick, depth, Pn, t_cache - size, t_cache))) {
            ++my_pruned;
            ++my_lex;
            level_ok = false;
          }
        }
      }
      // a tie node (one more colour class empties R): searched in id order, or put back
      if (level_ok && tie_ok && size < t_cache && 2 * (t_cache - size) >= popc<W>(Pn, wa)) {
        unsigned long long cls[W], R2[W];
#pragma unroll
        for (int q = 0; q < W; ++q) {
          cls[q] = R[q];
          R2[q] = R[q];
        }
        colour_class<W>(cls, R2, rows, wa, my_words);
        if (!any<W>(R2, wa) && tie_node(depth, Pn, size)) level_ok = false;
      }
      if (level_ok) {
        // the stack keeps only the record's live words (q < wa); reads mask the rest
#pragma unroll
        for (int q = 0; q < W; ++q)
          if (q < wa) {
            stkP[depth][q] = Pn[q];
            stkR[depth][q] = R[q];
          }
        if (cx.maximal)
#pragma unroll
          for (int q = 0; q < W; ++q)
            if (q < wa) stkX[depth][q] = Xn[q];
      }
    }
    if (level_ok) {
      unsigned long long R[W];
#pragma unroll
      for (int q = 0; q < W; ++q) R[q] = q < wa ? stkR[depth][q] : 0ull;
      const int u = highest<W>(R, wa);
      if (u >= 0) {
        // branching on u changes one word of the level: write only that word back
        const int qu = u >> 6;
        const unsigned long long ubit = 1ull << (u & 63);
        stkR[depth][qu] &= ~ubit;
        stkP[depth][qu] &= ~ubit;
        unsigned long long rem[W];
#pragma unroll
        for (int q = 0; q < W; ++q) rem[q] = q < wa ? stkP[depth][q] : 0ull;
        and_live<W>(Pn, rem, rows + u * W, wa);
        my_words += wa;
        if (cx.maximal) {
#pragma unroll
          for (int q = 0; q < W; ++q)
            Xn[q] = q < wa ? (stkX[depth][q] & rows[u * W + q]) : 0ull;
          stkX[depth][qu] |= ubit;
        }
        if (lex) lowc[depth + 1] = lowc[depth] | (uint8_t)((lowm[u >> 6] >> (u & 63)) & 1ull);
        ++depth;
        pick[depth] = (uint16_t)u;
        visit_node(depth, Pn, Xn);
        fresh = true;
        continue;
      }
    }
    if (depth == base_depth) break;
    --depth;
  }
}

// One lane per task (dynamic assignment).
template <int W>
__global__ void __launch_bounds__(128, 6) k_clique_tasks(Ctx cx, WideStore ws,
                                                      const WTask* __restrict__ in, int64_t nin,
                                                      unsigned long long* next) {
  unsigned long long my_exp = 0, my_pruned = 0, my_words = 0, my_lex = 0;
  bool limit_hit = false, out_of_time = false;
  int32_t t_cache = ld_volatile(&cx.st->tau);
  while (!out_of_time) {
    int64_t t = (int64_t)atomicAdd(next, 1ull);
    if (t >= nin) break;
    if (past_deadline(cx)) {
      atomicOr(&cx.st->err, 4);
      break;
    }
    const WTask& T = in[t];
    if (T.slot < 0) continue;
    uint16_t pick[MAXD + 1];
    {
      int d = 0;
#pragma unroll
      for (int q = 0; q < KWIDE; ++q) {
        unsigned long long c = T.C[q];
        while (c) {
          pick[d++] = (uint16_t)(q * 64 + __ffsll((long long)c) - 1);
          c &= c - 1;
        }
      }
    }
    unsigned long long Pn[W], Xn[W];
#pragma unroll
    for (int q = 0; q < W; ++q) {
      Pn[q] = T.P[q];
      Xn[q] = cx.maximal ? T.X[q] : 0ull;
    }
    t_cache = ld_volatile(&cx.st->tau);
    dense_node<W>(cx, ws, T.slot, T.depth, pick, Pn, Xn, true, T.cont, t_cache, my_exp,
                  my_pruned, my_words, my_lex, limit_hit, out_of_time);
  }
  if (limit_hit) atomicOr(&cx.st->err, 1);
  for (int o = 16; o; o >>= 1) {
    my_exp += __shfl_xor_sync(0xffffffffu, my_exp, o);
    my_pruned += __shfl_xor_sync(0xffffffffu, my_pruned, o);
    my_words += __shfl_xor_sync(0xffffffffu, my_words, o);
    my_lex += __shfl_xor_sync(0xffffffffu, my_lex, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(&cx.st->expansions, my_exp);
    atomicAdd(&cx.st->pruned, my_pruned);
    atomicAdd(&cx.st->tail_words, my_words);
    atomicAdd(&cx.st->lex_pruned, my_lex);
  }
}

template <int W>
__global__ void __launch_bounds__(KCfg<W>::WARPS * 32)
    k_clique_expand(Ctx cx, const Rec* __restrict__ in, const int32_t* __restrict__ seeds,
                    int64_t nin, WideStore ws) {
  constexpr int NW = KCfg<W>::WARPS;
  constexpr int BMW = 64 * W;   // candidates the bitmap tail handles
  __shared__ int32_t sP[NW][PSMEM];
  __shared__ int32_t sV[NW][MAXD];
  __shared__ uint16_t sOrd[NW][BMW], sPos[NW][BMW], sCol[NW][BMW];
  __shared__ int32_t sCnt[NW][BMW];
  __shared__ uint16_t sPerm[NW][BMW], sInv[NW][BMW];
  __shared__ int32_t sTot[NW], sNext[NW];
  __shared__ unsigned long long sAlive[NW][W];     // core filter: candidates kept
  // wide records (512 < |P| <= 1024, narrow instantiation only): degrees and colouring order
  constexpr int NWC = W == 1 ? NW : 1;
  constexpr int CBR = W == 1 ? CB_ROWS : 1;
  __shared__ uint16_t sCbDeg[NWC][CBR], sCbRem[NWC][CBR];
  extern __shared__ unsigned long long dynrows[];  // NW * BMW * W words: adjacency rows of P

  const int lane = threadIdx.x & 31;
  const int w = threadIdx.x >> 5;
  const unsigned FULL = 0xffffffffu;
  const DevGraph& g = cx.g;
  const int64_t gwarp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  int32_t* scratch = cx.pscratch ? cx.pscratch + gwarp * cx.pscratch_stride : nullptr;
  unsigned long long* rows = dynrows + (size_t)w * BMW * W;  // row i = rows[i*W .. i*W+W)

  unsigned long long my_exp = 0, my_pruned = 0, my_deq = 0, my_bytes = 0;

  while (true) {
    int64_t item = 0;
    __syncwarp();  // every lane is done with the previous record's shared state
    if (lane == 0) {
      item = (int64_t)atomicAdd((unsigned long long*)&cx.st->work_next, 1ull);
      if (item < nin && past_deadline(cx)) {
        atomicOr(&cx.st->err, 4);
        item = nin;
      }
    }
    item = __shfl_sync(FULL, item, 0);
    if (item >= nin) break;

    // ---- load the record ----
    int nv;
    if (seeds) {
      nv = 1;
      if (lane == 0) sV[w][0] = seeds[item];
    } else {
      nv = in[item].nv;
      if (nv < 1 || nv > MAXD) {  // not a record: reported, never followed
        if (lane == 0) {
          cx.st->bad_nv = nv;
          cx.st->bad_item = item;
          atomicOr(&cx.st->err, 8);
        }
        continue;
      }
      for (int i = lane; i < nv; i += 32) sV[w][i] = in[item].V[i];
    }
    __syncwarp();
    {
      // members: ranks of the graph in increasing order
      bool ok = true;
      for (int i = lane; i < nv; i += 32) {
        const int32_t v = sV[w][i];
        ok = ok && v >= 0 && v < g.n && (i == 0 || sV[w][i - 1] < v);
      }
      if (!__all_sync(FULL, ok)) {
        if (lane == 0) {
          cx.st->bad_nv = nv;
          cx.st->bad_item = item;
          atomicOr(&cx.st->err, 8);
        }
        continue;
      }
    }
    if (lane == 0) ++my_deq;

    // ---- candidate set P (ranks after every member, adjacent to all members) ----
    const int32_t* P;
    int p;
    {
      int32_t last = sV[w][nv - 1];
      int64_t b = g.ooff[last], e = g.ooff[last + 1];
      if (nv == 1) {
        P = g.oout + b;
        p = (int)(e - b);
        if (lane == 0) my_bytes += 4ull * (unsigned long long)p;
      } else {
        // candidates from the shortest member row (restricted to ranks > last)
        int64_t cb = b, ce = e;
        int srci = nv - 1;
        for (int i = 0; i < nv - 1; ++i) {
          int32_t v = sV[w][i];
          int64_t rb = g.ooff[v], re = g.ooff[v + 1];
          rb = lower_bound_dev64(g.oout, rb, re, last + 1);
          if (re - rb < ce - cb) {
            cb = rb;
            ce = re;
            srci = i;
          }
        }
        int32_t* dst = (ce - cb) <= PSMEM ? sP[w] : scratch;
        int cnt = 0;
        for (int64_t base = cb; base < ce; base += 32) {
          if (((base - cb) & 4095) == 4064) {  // a long row: stop at the deadline (uniform)
            int late = lane == 0 && past_deadline(cx);
            if (__shfl_sync(FULL, late, 0)) {
              if (lane == 0) atomicOr(&cx.st->err, 4);
              break;
            }
          }
          int64_t t = base + lane;
          bool keep = false;
          int32_t x = 0;
          if (t < ce) {
            x = __ldg(g.oout + t);
            keep = true;
            for (int i = 0; i < nv && keep; ++i) {
              if (i == srci) continue;  // the row the candidates come from
              int32_t v = sV[w][i];
              keep = contains64(g.oout, g.ooff[v], g.ooff[v + 1], x);
            }
          }
          unsigned bal = __ballot_sync(FULL, keep);
          if (keep) dst[cnt + __popc(bal & ((1u << lane) - 1))] = x;
          cnt += __popc(bal);
        }
        __syncwarp();
        if (lane == 0) my_bytes += 4ull * (unsigned long long)(ce - cb) * nv;
        P = dst;
        p = cnt;
      }
    }

    // ---- dequeue: prune (dominated), then result insertion ----
    const int32_t tau = warp_load(&cx.st->tau);  // one value for the warp's branches
    int bound = nv + p;
    if (!cx.no_prune && bound < tau) {
      if (lane == 0) ++my_pruned;
      continue;
    }
    if (nv >= MAXD && p > 0) {
      if (lane == 0) atomicOr(&cx.st->err, 1);
      continue;
    }
    // a record for the wide bitmap tail goes to its list untouched (dequeued there)
    const int lim = BMW < cx.split_above ? BMW : cx.split_above;  // bitmap tail limit here
    if (W == 1 && p > lim && p <= 64 * KWIDE && p <= cx.split_above) {
      if (lane == 0) {
        const int tier = p <= 128 ? 2 : (p <= 256 ? 1 : 0);  // 2, 4 or 8 words a row
        int64_t* cnt = tier == 2 ? &cx.st->small_count
                                 : (tier == 1 ? &cx.st->mid_count : &cx.st->wide_count);
        int64_t ds = (int64_t)atomicAdd((unsigned long long*)cnt, 1ull);
        Rec* r = (tier == 2 ? cx.small : (tier == 1 ? cx.mid : cx.wide)) + ds;
        r->nv = nv;
        r->bound = bound;
        for (int i = 0; i < nv; ++i) r->V[i] = sV[w][i];
        --my_deq;
      }
      continue;
    }
    // a record too wide for the bitmap tiers (512 < |P| <= 1024) is first coloured greedily on
    // an adjacency bitmap of P (global scratch): if the colours do not lift it to tau, no
    // clique below it can, and it is dropped before its children are created
    if (W == 1 && cx.cbits && !cx.no_prune && p > 64 * KWIDE && p <= CB_ROWS && nv < tau) {
      unsigned long long* cb = cx.cbits + gwarp * (int64_t)CB_ROWS * CB_W;
      const int cw = (p + 63) >> 6;
      for (int64_t i = lane; i < (int64_t)p * CB_W; i += 32) cb[i] = 0ull;
      __syncwarp();
      const int32_t plast = P[p - 1];
      for (int i = 0; i < p; ++i) {
        const int32_t pi = P[i];
        const int64_t rb = g.ooff[pi], re = g.ooff[pi + 1];
        for (int64_t t = rb + lane; t < re; t += 32) {
          const int32_t x = __ldg(g.oout + t);
          if (x > plast) continue;
          const int j = lower_bound_dev(P, i + 1, p, x);  // out-neighbours rank above pi
          if (j < p && P[j] == x) {
            atomicOr(&cb[(int64_t)i * CB_W + (j >> 6)], 1ull << (j & 63));
            atomicOr(&cb[(int64_t)j * CB_W + (i >> 6)], 1ull << (i & 63));
          }
        }
      }
      __syncwarp();
      // greedy colouring of P with the candidates in order of degree (highest first: the
      // initial order of colour-ordered clique search, which tightens the bound), one colour
      // class at a time, warp-cooperative: the warp scans the uncoloured candidates 32 at a
      // time, the first one not adjacent to the class joins it and the others are re-tested
      // against it.  Candidates with fewer than need - 1 neighbours in P cannot be in a clique
      // reaching tau and are left out.
      int drop = 0;
      if constexpr (W == 1) {
        const int need = tau - nv;  // colours the record needs to reach tau
        uint16_t* deg = sCbDeg[w];
        uint16_t* rem = sCbRem[w];  // uncoloured candidates, by degree
        int alive = 0;
        for (int i = lane; i < p; i += 32) {
          int d = 0;
          for (int q = 0; q < cw; ++q) d += __popcll(cb[(int64_t)i * CB_W + q]);
          deg[i] = (uint16_t)d;
          alive += d >= need - 1 ? 1 : 0;
        }
        for (int o = 16; o; o >>= 1) alive += __shfl_xor_sync(FULL, alive, o);
        __syncwarp();
        if (alive < need) {
          drop = 1;
        } else {
          for (int i = lane; i < p; i += 32) {
            const int di = deg[i];
            if (di < need - 1) continue;
            int r = 0;
            for (int j = 0; j < p; ++j) {
              const int dj = deg[j];
              r += (dj >= need - 1 && (dj > di || (dj == di && j < i))) ? 1 : 0;
            }
            rem[r] = (uint16_t)i;
          }
          __syncwarp();
          int nrem = alive, colours = 0;
          while (nrem > 0 && colours < need) {
            ++colours;
            unsigned long long forb = 0ull;  // lane q < cw: word q of the class's neighbours
            int out = 0;
            for (int base = 0; base < nrem; base += 32) {
              const int t = base + lane;
              const int v = t < nrem ? (int)rem[t] : 0;
              const unsigned long long fw = __shfl_sync(FULL, forb, (v >> 6) & 31);
              bool cand = t < nrem && !((fw >> (v & 63)) & 1ull);
              bool joined = false;
              unsigned m = __ballot_sync(FULL, cand);
              while (m) {
                const int src = __ffs(m) - 1;
                const int u = __shfl_sync(FULL, v, src);
                const unsigned long long* row = cb + (int64_t)u * CB_W;
                if (lane < cw) forb |= row[lane];
                if (lane == src) {
                  cand = false;
                  joined = true;
                } else if (cand) {
                  cand = !((row[v >> 6] >> (v & 63)) & 1ull);
                }
                m = __ballot_sync(FULL, cand);
              }
              const bool stay = t < nrem && !joined;
              const unsigned sm = __ballot_sync(FULL, stay);
              __syncwarp();  // every lane holds its entry before the compaction writes
              if (stay) rem[out + __popc(sm & ((1u << lane) - 1))] = (uint16_t)v;
              out += __popc(sm);
              __syncwarp();
            }
            nrem = out;
          }
          drop = (nrem == 0 && colours < need) ? 1 : 0;  // |V| + colours < tau
        }
        if (drop && lane == 0) ++my_pruned;
      }
      if (drop) continue;
    }
    // a record that must be split reserves its children's staging slots first; if the
    // staging array is full it goes back to the frontier untouched (re-dequeued later)
    int64_t base_slot = 0;
    if (p > lim) {
      bool reserved = true;
      if (lane == 0) {
        base_slot = (int64_t)atomicAdd((unsigned long long*)&cx.st->stage_count,
                                       (unsigned long long)p);
        if (base_slot + p > cx.stage_cap) {
          reserved = false;
          int64_t ds = (int64_t)atomicAdd((unsigned long long*)&cx.st->defer_count, 1ull);
          Rec* r = cx.deferred + ds;
          r->nv = nv;
          r->bound = bound;
          for (int i = 0; i < nv; ++i) r->V[i] = sV[w][i];
          --my_deq;
        }
      }
      reserved = __shfl_sync(FULL, (int)reserved, 0);
      base_slot = __shfl_sync(FULL, base_slot, 0);
      if (!reserved) continue;
    }
    if (lane == 0 && nv >= tau) {
      bool rel = true;
      if (cx.maximal) rel = (p == 0) && is_maximal(g, sV[w], nv);
      if (rel) add_result(cx, sV[w], nv, 0, nullptr);
    }
    if (p == 0) continue;

    if (p <= lim) {
      // ================= bitmap tail: finish the whole subtree in this warp =================
      // Colour-ordered branching (the MCQ/MCS scheme of exact maximum-clique search): a
      // greedy colouring of the candidates P bounds the clique they can add by the number of
      // colours; children are taken from the highest colour class down and every remaining
      // child is pruned once |C| + colours(remaining) < tau.  Every clique is still produced
      // exactly once: after a child v is explored, v leaves the candidates of its siblings.
      const int wa = (p + 63) >> 6;  // words in use
      int32_t* sp = sP[w];
      if (P != sp) {
        for (int i = lane; i < p; i += 32) sp[i] = P[i];
        __syncwarp();
      }
      const int32_t plast = sp[p - 1];
      // Candidates are re-indexed by their degree inside P, highest first (the initial order
      // of colour-ordered clique search: it tightens the greedy colouring).  A first scan counts
      // the degrees, a counting sort gives the order, a second scan builds the rows.
      int32_t* dg = sCnt[w];
      uint16_t* perm = sPerm[w];  // new index -> index in sp
      uint16_t* inv = sInv[w];    // index in sp -> new index
      for (int i = lane; i < p; i += 32) dg[i] = 0;
      __syncwarp();
      // candidates a clique reaching tau needs below this record (0: no core filter)
      int core_need = 0;
      if (!cx.no_prune) {
        const int32_t t_now = warp_load(&cx.st->tau);  // core_need steers warp-wide code
        if (t_now != INT32_MIN && t_now - nv > 1) core_need = t_now - nv;
      }
      // candidates inside the core bitmap (the last ranks of the order): rows come from bit
      // tests of the bitmap, every (candidate, 32 candidates) step independent of the others
      const bool in_core = g.core_bits != nullptr && sp[0] >= g.core_base;
      int pass = 0;
      for (; pass < 2; ++pass) {
        if (pass == 1) {
          for (int i = lane; i < p * W; i += 32) rows[i] = 0;
          __syncwarp();
        }
        if (in_core) {
          // each lane owns whole rows: candidate i's bits against every candidate j (the
          // loads of one row are independent and cached), the row built in registers
          const int cw = g.core_n >> 6;
          for (int i = lane; i < p; i += 32) {
            const unsigned long long* crow =
                g.core_bits + (int64_t)(sp[i] - g.core_base) * cw;
            if (pass == 0) {
              int d = 0;
              for (int j = 0; j < p; ++j) {
                const int x = sp[j] - g.core_base;
                d += (j != i && ((__ldg(crow + (x >> 6)) >> (x & 63)) & 1ull)) ? 1 : 0;
              }
              dg[i] = d;
            } else {
              unsigned long long r[W];
#pragma unroll
              for (int q = 0; q < W; ++q) r[q] = 0ull;
              for (int j = 0; j < p; ++j) {
                const int x = sp[j] - g.core_base;
                if (j != i && ((__ldg(crow + (x >> 6)) >> (x & 63)) & 1ull)) set_bit<W>(r, inv[j]);
              }
              const int a = inv[i];
#pragma unroll
              for (int q = 0; q < W; ++q) rows[a * W + q] = r[q];
            }
          }
          if (lane == 0) my_bytes += 4ull * (unsigned long long)p * ((p + 31) >> 5);
        }
        for (int i = 0; i < p && !in_core; ++i) {
          int32_t v = sp[i];
          int64_t rb = g.ooff[v], re = g.ooff[v + 1];
          int64_t scanned = 0;
          for (int64_t base = rb; base < re; base += 32) {
            int64_t t = base + lane;
            int32_t x = t < re ? __ldg(g.oout + t) : INT32_MAX;
            if (x <= plast) {
              int j = lower_bound_dev(sp, i + 1, p, x);
              if (j < p && sp[j] == x) {
                if (pass == 0) {
                  atomicAdd(dg + i, 1);
                  atomicAdd(dg + j, 1);
                } else {
                  int a = inv[i], b = inv[j];
                  atomicOr(rows + a * W + (b >> 6), 1ull << (b & 63));
                  atomicOr(rows + b * W + (a >> 6), 1ull << (a & 63));
                }
              }
            }
            scanned += 32;
            if (__all_sync(FULL, x > plast)) break;  // rows are sorted
          }
          if (lane == 0) my_bytes += 4ull * (unsigned long long)(scanned < re - rb ? scanned : re - rb);
        }
        __syncwarp();
        if (pass == 0 && core_need > 1) {
          // a clique of size >= tau below this record has at least core_need = tau - |V|
          // members in P, each with at least core_need - 1 neighbours in P: with fewer such
          // candidates the record holds no result (the record itself was handled above)
          int c = 0;
          for (int i = lane; i < p; i += 32) c += dg[i] >= core_need - 1 ? 1 : 0;
          for (int o = 16; o; o >>= 1) c += __shfl_xor_sync(FULL, c, o);
          if (c < core_need) break;
        }
        if (pass == 0 && lane == 0) {
          // counting sort by degree, descending (ties: lower index first)
          uint16_t* bucket = sCol[w];
          for (int d = 0; d < p; ++d) bucket[d] = 0;
          for (int i = 0; i < p; ++i) ++bucket[dg[i]];
          int at = 0;
          for (int d = p - 1; d >= 0; --d) {
            int c = bucket[d];
            bucket[d] = (uint16_t)at;
            at += c;
          }
          for (int i = 0; i < p; ++i) {
            int a = bucket[dg[i]]++;
            perm[a] = (uint16_t)i;
            inv[i] = (uint16_t)a;
          }
        }
        __syncwarp();
      }
      if (pass < 2) {  // rejected by the degree count
        if (lane == 0) ++my_pruned;
        continue;
      }
      // core filter on the rows: candidates with fewer than core_need - 1 neighbours among the
      // remaining ones cannot be in a clique reaching tau; they are removed (rows cleared, bits
      // dropped from every row) until every remaining candidate has enough, and the record is
      // dropped if fewer than core_need remain.  Removed candidates stay as isolated vertices:
      // their colour bound (|V| + 1 < tau) prunes them at once.
      if (core_need > 1) {
        const int alive = core_peel<W>(rows, p, core_need, sAlive[w], lane);
        if (alive < core_need) {
          if (lane == 0) ++my_pruned;
          continue;
        }
      }
      // record-level colouring (index order) and the order of the children by colour
      uint16_t* ord = sOrd[w];   // vertices by ascending colour
      uint16_t* pos = sPos[w];   // position of each vertex in ord
      uint16_t* col = sCol[w];   // colour of each vertex (1-based)
      if (lane == 0) {
        unsigned long long left[W];
#pragma unroll
        for (int q = 0; q < W; ++q) left[q] = 0;
        for (int i = 0; i < p; ++i) set_bit<W>(left, i);
        int c = 0, o = 0;
        while (any<W>(left, wa)) {
          ++c;
          unsigned long long cls[W];
#pragma unroll
          for (int q = 0; q < W; ++q) cls[q] = left[q];
          int v;
          while ((v = lowest<W>(cls, wa)) >= 0) {
#pragma unroll
            for (int q = 0; q < W; ++q) cls[q] &= ~rows[v * W + q];
            clear_bit<W>(cls, v);
            clear_bit<W>(left, v);
            col[v] = (uint16_t)c;
            pos[v] = (uint16_t)o;
            ord[o++] = (uint16_t)v;
          }
        }
      }
      __syncwarp();
      bool limit_hit = false, out_of_time = false;
      if constexpr (W > 1) {
        // dense record: keep its bitmap in a store slot and queue its children as tasks
        int32_t t_cache = ld_volatile(&cx.st->tau);
        int slot = 0;
        if (lane == 0) slot = (int)atomicAdd(ws.nslots, 1ull);
        slot = __shfl_sync(FULL, slot, 0);
        unsigned long long* grow = ws.rows + (int64_t)slot * BMW * W;
        for (int i = lane; i < p * W; i += 32) grow[i] = rows[i];
        for (int a = lane; a < p; a += 32) ws.vmap[(int64_t)slot * BMW + a] = sp[perm[a]];
        for (int a = lane; a < nv; a += 32) ws.recV[(int64_t)slot * MAXD + a] = sV[w][a];
        if (lane == 0) {
          ws.recN[slot] = nv;
          ws.recP[slot] = p;
        }
        if (ws.cid) {
          // ids of the candidates, their order by id (rank by counting), the record's ids
          int32_t* cid = ws.cid + (int64_t)slot * BMW;
          for (int a = lane; a < p; a += 32) cid[a] = __ldg(g.vert_of + sp[perm[a]]);
          __syncwarp();
          for (int a = lane; a < p; a += 32) {
            const int32_t x = cid[a];
            int r = 0;
            for (int b2 = 0; b2 < p; ++b2) r += cid[b2] < x ? 1 : 0;
            ws.byid[(int64_t)slot * BMW + r] = (uint16_t)a;
          }
          int32_t* rid = ws.rid + (int64_t)slot * MAXD;
          for (int a = lane; a < nv; a += 32) {
            const int32_t x = __ldg(g.vert_of + sV[w][a]);
            int r = 0;
            for (int b2 = 0; b2 < nv; ++b2) r += __ldg(g.vert_of + sV[w][b2]) < x ? 1 : 0;
            rid[r] = x;
          }
        }
        __threadfence_block();
        __syncwarp();
        for (int i = p - 1 - lane; i >= 0 && !out_of_time; i -= 32) {
          const int v0 = ord[i];
          if (!cx.no_prune && nv + (int)col[v0] < t_cache) {
            ++my_pruned;
            continue;
          }
          unsigned long long Pi[W], Xi[W];
#pragma unroll
          for (int q = 0; q < W; ++q) {
            Pi[q] = 0;
            Xi[q] = 0;
          }
          for (int u = 0; u < p; ++u) {
            if ((rows[v0 * W + (u >> 6)] & (1ull << (u & 63))) == 0) continue;
            if (pos[u] < i) set_bit<W>(Pi, u);
            else set_bit<W>(Xi, u);
          }
          unsigned long long qs = atomicAdd(ws.q_count, 1ull);
          if ((int64_t)qs < ws.q_cap) {
            WTask* t = ws.q_out + qs;
            t->slot = slot;
            t->depth = 0;
            t->cont = 0;
            const uint16_t pk0 = (uint16_t)v0;
            write_picks(t, &pk0, 0);
#pragma unroll
            for (int q = 0; q < KWIDE; ++q) {
              t->P[q] = q < W ? Pi[q] : 0ull;
              if (cx.maximal) t->X[q] = q < W ? Xi[q] : 0ull;
            }
          } else {
            uint16_t pk[MAXD + 1];
            pk[0] = (uint16_t)v0;
            unsigned long long words_here = 0, lex_here = 0;  // counted for the task kernel
            dense_node<W>(cx, ws, slot, 0, pk, Pi, Xi, false, 0, t_cache, my_exp,
                          my_pruned, words_here, lex_here, limit_hit, out_of_time);
          }
        }
      } else {
      // Two-level lane tasks, both in colour order (the MCQ scheme).  Children: ord[i] for i
      // from p-1 down, with the candidates adjacent to it that come earlier in ord (P_i), the
      // explored ones later in ord (X_i) and the bound |V| + colour(ord[i]).  Grandchildren of
      // child i: the members of P_i in the colour order of a greedy colouring of P_i (colour
      // classes in turn, members of a class by index), taken from the last; grandchild j has
      // the members of P_i before it (adjacent to j) as candidates, those after it as explored,
      // and the bound |V| + 1 + colour_i(j).  Phase 1 visits every child node and counts its
      // viable grandchildren; phase 2 hands one grandchild subtree at a time to a lane through
      // a shared counter.  Every clique of the record's subtree is visited exactly once.
      int32_t t_cache = ld_volatile(&cx.st->tau);
      int32_t* cnt = sCnt[w];
      auto child_sets = [&](int i, unsigned long long* Pi, unsigned long long* Xi) {
        const int v0 = ord[i];
#pragma unroll
        for (int q = 0; q < W; ++q) {
          Pi[q] = 0;
          Xi[q] = 0;
        }
        for (int u = 0; u < p; ++u) {
          if ((rows[v0 * W + (u >> 6)] & (1ull << (u & 63))) == 0) continue;
          if (pos[u] < i) set_bit<W>(Pi, u);
          else set_bit<W>(Xi, u);
        }
      };
      // greedy colouring of S in index order: calls f(v, colour) for every member in the
      // colour order; stops early when f returns false
      auto colour_walk = [&](const unsigned long long* S, auto&& f) {
        unsigned long long left[W];
#pragma unroll
        for (int q = 0; q < W; ++q) left[q] = S[q];
        int c = 0;
        while (any<W>(left, wa)) {
          ++c;
          unsigned long long cls[W];
#pragma unroll
          for (int q = 0; q < W; ++q) cls[q] = left[q];
          int v;
          while ((v = lowest<W>(cls, wa)) >= 0) {
#pragma unroll
            for (int q = 0; q < W; ++q) cls[q] &= ~rows[v * W + q];
            clear_bit<W>(cls, v);
            clear_bit<W>(left, v);
            if (!f(v, c)) return;
          }
        }
      };
      // ---- phase 1: the child nodes ----
      for (int i = p - 1 - lane; i >= 0; i -= 32) {
        const int v0 = ord[i];
        cnt[i] = 0;
        if (!cx.no_prune && nv + (int)col[v0] < t_cache) {
          ++my_pruned;
          continue;
        }
        unsigned long long Pi[W], Xi[W];
        child_sets(i, Pi, Xi);
        ++my_exp;
        const int size = nv + 1;
        if (size >= t_cache) {
          bool rel = true;
          if (cx.maximal) {
            if (any<W>(Pi, wa) || any<W>(Xi, wa)) rel = false;
            else {
              int32_t C[MAXD];
              for (int a = 0; a < nv; ++a) C[a] = sV[w][a];
              C[nv] = sp[perm[v0]];
              rel = is_maximal(g, C, size);
            }
          }
          if (rel) {
            int32_t pr = sp[perm[v0]];
            add_result(cx, sV[w], nv, 1, &pr);
            t_cache = ld_volatile(&cx.st->tau);
          }
        }
        if (any<W>(Pi, wa) && size >= MAXD) {
          limit_hit = true;
          continue;
        }
        // viable grandchildren: colour_i(j) >= tau - |V| - 1
        const int cmin = (cx.no_prune || t_cache == INT32_MIN) ? 0 : t_cache - nv - 1;
        int viable = 0;
        colour_walk(Pi, [&](int, int c) {
          if (c >= cmin) ++viable;
          return true;
        });
        cnt[i] = viable;
      }
      __syncwarp();
      if (lane == 0) {
        int acc = 0;
        for (int i = 0; i < p; ++i) {
          int c = cnt[i];
          cnt[i] = acc;  // exclusive prefix
          acc += c;
        }
        sTot[w] = acc;
        sNext[w] = 0;
      }
      __syncwarp();
      const int ntask = sTot[w];
      // per-lane DFS stack: the untried candidates (and, for maximality, the explored ones)
      // of every level; pick[d] = index in P of the vertex added at depth d
      unsigned long long stkP[MAXD][W];
      unsigned long long stkR[MAXD][W];
      unsigned long long stkX[MAXD][W];
      uint16_t pick[MAXD + 1];
      // ---- phase 2: grandchild subtrees, taken dynamically ----
      while (!out_of_time) {
        int t = atomicAdd(&sNext[w], 1);
        if (t >= ntask) break;
        // child i: the last index with cnt[i] <= t (cnt is non-decreasing)
        int lo = 0, hi = p - 1;
        while (lo < hi) {
          int mid = (lo + hi + 1) >> 1;
          if (cnt[mid] <= t) lo = mid;
          else hi = mid - 1;
        }
        const int i = lo;
        const int k = t - cnt[i];  // the k-th grandchild from the end of the colour order
        unsigned long long Pi[W], Xn[W];
        child_sets(i, Pi, Xn);
        const int total = popc<W>(Pi, wa);
        const int target = total - 1 - k;  // position of the grandchild in the colour order
        // the grandchild j, the members before it (prefix) and its colour
        unsigned long long prefix[W];
#pragma unroll
        for (int q = 0; q < W; ++q) prefix[q] = 0;
        int j = -1, cj = 0, at = 0;
        colour_walk(Pi, [&](int v, int c) {
          if (at == target) {
            j = v;
            cj = c;
            return false;
          }
          set_bit<W>(prefix, v);
          ++at;
          return true;
        });
        const int depth0_size = nv + 2;
        if (j < 0 || (!cx.no_prune && nv + 1 + cj < ld_volatile(&cx.st->tau))) {
          ++my_pruned;  // tau rose since the count
          continue;
        }
        unsigned long long Pn[W];
#pragma unroll
        for (int q = 0; q < W; ++q) {
          Pn[q] = prefix[q] & rows[j * W + q];
          // explored: X_i, and the members of P_i after j
          Xn[q] = (Xn[q] | (Pi[q] & ~prefix[q])) & rows[j * W + q];
        }
        (void)depth0_size;
        int depth = 1;
        pick[0] = (uint16_t)ord[i];
        pick[1] = (uint16_t)j;
        // visit the node (record + picks[0..depth], candidates Pn, explored Xn), colour it once,
        // then branch over its high-colour set (as in dense_node: level d keeps the untried
        // candidates stkP, the untried high-colour ones stkR and the explored ones stkX)
        bool visit = true;
        while (true) {
          int size = nv + depth + 1;
          bool level_ok = true;
          if (visit) {
            ++my_exp;
            if ((my_exp & 31) == 0) {
              t_cache = ld_volatile(&cx.st->tau);
              if ((my_exp & 1023) == 0 && past_deadline(cx)) {
                atomicOr(&cx.st->err, 4);
                out_of_time = true;
                break;
              }
            }
            if (size >= t_cache) {
              bool rel = true;
              if (cx.maximal) {
                if (any<W>(Pn, wa) || any<W>(Xn, wa)) rel = false;
                else {
                  int32_t C[MAXD];
                  for (int a = 0; a < nv; ++a) C[a] = sV[w][a];
                  for (int d = 0; d <= depth; ++d) C[nv + d] = sp[perm[pick[d]]];
                  rel = is_maximal(g, C, size);
                }
              }
              if (rel) {
                int32_t pr[MAXD];
                for (int d = 0; d <= depth; ++d) pr[d] = sp[perm[pick[d]]];
                add_result(cx, sV[w], nv, depth + 1, pr);
                t_cache = ld_volatile(&cx.st->tau);
              }
            }
            visit = false;
            // colour once: R = the candidates left after classes 1 .. tau-|node|-1
            unsigned long long R[W];
#pragma unroll
            for (int q = 0; q < W; ++q) R[q] = Pn[q];
            level_ok = any<W>(R, wa);
            if (level_ok && size >= MAXD) {
              limit_hit = true;
              level_ok = false;
            }
            if (level_ok && !cx.no_prune && size + popc<W>(R, wa) < t_cache) {
              ++my_pruned;  // |V| + |P| < tau: no colouring needed
              level_ok = false;
            }
            if (level_ok && !cx.no_prune && size < t_cache) {
              const int kmin = t_cache - size;
              for (int c = 1; c < kmin && any<W>(R, wa); ++c) {
                unsigned long long cls[W];
#pragma unroll
                for (int q = 0; q < W; ++q) cls[q] = R[q];
                int v;
                while ((v = lowest<W>(cls, wa)) >= 0) {
#pragma unroll
                  for (int q = 0; q < W; ++q) cls[q] &= ~rows[v * W + q];
                  clear_bit<W>(cls, v);
                  clear_bit<W>(R, v);
                }
              }
              if (!any<W>(R, wa)) {
                ++my_pruned;
                level_ok = false;
              }
            }
            if (level_ok) {
#pragma unroll
              for (int q = 0; q < W; ++q) {
                stkP[depth][q] = Pn[q];
                stkR[depth][q] = R[q];
              }
              if (cx.maximal)
#pragma unroll
                for (int q = 0; q < W; ++q) stkX[depth][q] = Xn[q];
            }
          }
          if (level_ok) {
            unsigned long long R[W];
#pragma unroll
            for (int q = 0; q < W; ++q) R[q] = stkR[depth][q];
            const int u = highest<W>(R, wa);
            if (u >= 0) {
              // child: add u; its candidates are this node's untried ones adjacent to u
              unsigned long long rem[W];
#pragma unroll
              for (int q = 0; q < W; ++q) rem[q] = stkP[depth][q];
              clear_bit<W>(R, u);
              clear_bit<W>(rem, u);
#pragma unroll
              for (int q = 0; q < W; ++q) {
                stkR[depth][q] = R[q];
                stkP[depth][q] = rem[q];
                Pn[q] = rem[q] & rows[u * W + q];
              }
              if (cx.maximal) {  // the explored set only matters for maximality
                unsigned long long xs[W];
#pragma unroll
                for (int q = 0; q < W; ++q) {
                  xs[q] = stkX[depth][q];
                  Xn[q] = xs[q] & rows[u * W + q];
                }
                set_bit<W>(xs, u);
#pragma unroll
                for (int q = 0; q < W; ++q) stkX[depth][q] = xs[q];
              }
              ++depth;
              pick[depth] = (uint16_t)u;
              visit = true;
              continue;
            }
          }
          // done with this node: back to its parent
          if (depth == 1) break;
          --depth;
        }
      }
      }
      if (limit_hit) atomicOr(&cx.st->err, 1);
      __syncwarp();
      continue;
    }

    // ================= split: one child per d in P, pushed to the staging array =================
    const int32_t plast = P[p - 1];
    for (int j = 0; j < p; ++j) {
      if ((j & 63) == 63) {  // a long record: stop at the deadline (uniform)
        int late = lane == 0 && past_deadline(cx);
        if (__shfl_sync(FULL, late, 0)) {
          if (lane == 0) atomicOr(&cx.st->err, 4);
          break;
        }
      }
      int32_t d = P[j];
      int64_t rb = g.ooff[d], re = g.ooff[d + 1];
      int64_t re2 = lower_bound_dev64(g.oout, rb, re, plast + 1);
      int alen = p - j - 1;
      int64_t blen = re2 - rb;
      int c = 0;
      if (alen > 0 && blen > 0) {
        if (blen <= alen) {
          for (int64_t t0 = rb; t0 < re2; t0 += 32) {
            int64_t t = t0 + lane;
            bool hit = false;
            if (t < re2) {
              int32_t x = __ldg(g.oout + t);
              int q = lower_bound_dev(P, j + 1, p, x);
              hit = q < p && P[q] == x;
            }
            c += __popc(__ballot_sync(FULL, hit));
          }
        } else {
          for (int t0 = j + 1; t0 < p; t0 += 32) {
            int t = t0 + lane;
            bool hit = false;
            if (t < p) hit = contains64(g.oout, rb, re2, P[t]);
            c += __popc(__ballot_sync(FULL, hit));
          }
        }
      }
      if (lane == 0) {
        ++my_exp;
        my_bytes += 4ull * (unsigned long long)(alen + blen);
        int32_t t_now = ld_volatile(&cx.st->tau);
        int cb = nv + 1 + c;
        if (!cx.no_prune && cb < t_now) {
          ++my_pruned;
        } else if (c == 0) {
          // a leaf: the child is a clique with no extension; it is dequeued at once
          ++my_deq;
          int size = nv + 1;
          if (size >= t_now) {
            bool rel = true;
            if (cx.maximal) {
              int32_t C[MAXD];
              for (int i = 0; i < nv; ++i) C[i] = sV[w][i];
              C[nv] = d;
              rel = is_maximal(g, C, size);
            }
            if (rel) add_result(cx, sV[w], nv, 1, &d);
          }
        } else {
          Rec* r = cx.stage + base_slot + j;
          r->nv = nv + 1;
          r->bound = cb;
          for (int i = 0; i < nv; ++i) r->V[i] = sV[w][i];
          r->V[nv] = d;
        }
      }
    }
    __syncwarp();
  }
  if (lane == 0) {
    atomicAdd(&cx.st->dequeued, my_deq);
    atomicAdd(&cx.st->adj_bytes, my_bytes);
  }
  // per-lane counters (lanes count bitmap-tail nodes)
  for (int o = 16; o; o >>= 1) {
    my_exp += __shfl_xor_sync(FULL, my_exp, o);
    my_pruned += __shfl_xor_sync(FULL, my_pruned, o);
  }
  if (lane == 0) {
    atomicAdd(&cx.st->expansions, my_exp);
    atomicAdd(&cx.st->pruned, my_pruned);
  }
}

// ---------------------------------------------------------------------------------------------
// frontier plumbing
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ int bucket_of(int32_t bound) { return bound >= NB - 1 ? NB - 1 : bound; }

// Seed key = (class << 24) | bound, bound = 1 + |N+(v)|.  Class 1: the candidate set fits the
// narrow bitmap tail (|N+(v)| <= 64).  Seeds are consumed class 1 first, each class in
// descending bound order: the narrow seeds are cheap and usually raise tau to its final
// value (planted or core cliques), so the wide, dense seeds are searched under a high tau.
// With a seed partition, seeds of other parts get key 0 (class 0, bound 0): they sort last and
// are never taken (every real seed's bound is at least 1).
__global__ void k_seed_bounds(DevGraph g, int32_t part_index, int32_t part_count, int32_t* keys,
                              int32_t* vals) {
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < g.n;
       r += (int64_t)gridDim.x * blockDim.x) {
    int32_t outdeg = (int32_t)(g.ooff[r + 1] - g.ooff[r]);
    const bool mine = part_count <= 1 || seed_part(g.vert_of[r], part_count) == part_index;
    keys[r] = mine ? (((outdeg <= 64 ? 1 : 0) << 24) | (1 + outdeg)) : 0;
    vals[r] = (int32_t)r;
  }
}

// Raise tau to at least v (a threshold another part of a partitioned query published).
__global__ void k_raise_tau(int32_t* tau, int32_t v) {
  if (threadIdx.x == 0 && blockIdx.x == 0) atomicMax(tau, v);
}

// Count one into hist[b] for every lane with b >= 0; lanes of a warp with the same bucket
// (neighbouring keys mostly share one) add together, one atomic per distinct bucket.
__device__ __forceinline__ void warp_hist_add(int32_t* hist, int b) {
  const unsigned peers = __match_any_sync(0xffffffffu, b);
  if (b >= 0 && (threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(&hist[b], __popc(peers));
}

__global__ void k_bucket_hist(const int32_t* keys, int64_t n, int32_t* hist) {
  // whole warps step together (the tail lanes pass b = -1)
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i0 = blockIdx.x * (int64_t)blockDim.x; i0 < n; i0 += stride) {
    const int64_t i = i0 + threadIdx.x;
    const int b = i < n ? (keys[i] >> 24) * NB + bucket_of(keys[i] & 0xffffff) : -1;
    warp_hist_add(hist, b);
  }
}

__global__ void k_stage_hist(const Rec* stage, int64_t cnt, int32_t* hist) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i0 = blockIdx.x * (int64_t)blockDim.x; i0 < cnt; i0 += stride) {
    const int64_t i = i0 + threadIdx.x;
    const int b = (i < cnt && stage[i].nv > 0) ? bucket_of(stage[i].bound) : -1;
    warp_hist_add(hist, b);
  }
}

// Are ranks a != b adjacent?  (the out-row of the lower rank holds the higher one)
__device__ __forceinline__ bool adjacent_rank(const DevGraph& g, int32_t a, int32_t b) {
  if (a > b) {
    const int32_t t = a;
    a = b;
    b = t;
  }
  return contains64(g.oout, g.ooff[a], g.ooff[a + 1], b);
}

// Warm start for tau (all-cliques ranking): one warp per seed grows a clique greedily inside
// the seed's candidates (narrow seeds, at most 64 candidates: in the order of their number of
// neighbours among the candidates, computed once -- ties: larger graph degree, then lower
// rank -- each one adjacent to all added before; wide seeds: always the remaining candidate
// of largest graph degree, then keeping the candidates adjacent to it) and publishes subset_tau of its size.  The cliques themselves
// are not recorded (the search finds them again); only the lower bound on the k-th best is
// used, so the answer is unchanged.  buf: max_out entries per warp.
__global__ void __launch_bounds__(256)
    k_greedy_tau(DevGraph g, const int32_t* __restrict__ seeds, int64_t nseeds, int32_t k,
                 int32_t* __restrict__ buf, int32_t* __restrict__ tau) {
  const int lane = threadIdx.x & 31;
  const unsigned FULL = 0xffffffffu;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  __shared__ int32_t sGP[8][64];              // narrow seeds: the candidates (8 warps a block)
  __shared__ unsigned long long sGRow[8][64];  // and their adjacency rows
  const int wl = threadIdx.x >> 5;
  int32_t* P = buf + warp * (int64_t)g.max_out;
  for (int64_t i = warp; i < nseeds; i += nwarps) {
    const int32_t v = seeds[i];
    const int64_t b = g.ooff[v];
    int p = (int)(g.ooff[v + 1] - b);
    for (int t = lane; t < p; t += 32) P[t] = g.oout[b + t];
    __syncwarp();
    int c = 1;
    if (p <= 64) {
      // narrow: candidates ordered once by (neighbours among the candidates, graph degree,
      // -rank); a 64-bit mask keeps the ones adjacent to every candidate added so far.  The
      // candidates' adjacency is built once as 64-bit rows in shared memory (each candidate's
      // out-row scanned by the warp, its entries located in P by binary search)
      int32_t* sp = sGP[wl];
      unsigned long long* rows = sGRow[wl];
      for (int t = lane; t < p; t += 32) sp[t] = P[t];
      for (int t = lane; t < 64; t += 32) rows[t] = 0ull;
      __syncwarp();
      const int32_t plast = sp[p - 1];
      for (int a = 0; a < p; ++a) {
        const int64_t rb = g.ooff[sp[a]], re = g.ooff[sp[a] + 1];
        for (int64_t b0 = rb; b0 < re; b0 += 32) {
          const int64_t t = b0 + lane;
          const int32_t y = t < re ? __ldg(g.oout + t) : INT32_MAX;
          if (y <= plast) {
            int lo = a + 1, hi = p;  // out-neighbours rank above sp[a]
            while (lo < hi) {
              const int mid = (lo + hi) >> 1;
              if (sp[mid] < y) lo = mid + 1;
              else hi = mid;
            }
            if (lo < p && sp[lo] == y) {
              atomicOr(&rows[a], 1ull << lo);
              atomicOr(&rows[lo], 1ull << a);
            }
          }
          if (__all_sync(FULL, y > plast)) break;  // rows are sorted
        }
      }
      __syncwarp();
      long long key[2] = {-1, -1};
      for (int h = 0; h < 2; ++h) {
        const int t = lane + 32 * h;
        if (t >= p) continue;
        const int32_t x = sp[t];
        const int inner = __popcll(rows[t]);
        const int32_t d = min(__ldg(g.deg + __ldg(g.vert_of + x)), 0xFFFFF);
        key[h] = ((long long)inner << 40) | ((long long)d << 20) |
                 (long long)(0xFFFFF - (x & 0xFFFFF));
      }
      unsigned long long alive = p == 64 ? ~0ull : ((1ull << p) - 1);
      while (alive) {
        long long bk = -1;
        int bt = -1;
        for (int h = 0; h < 2; ++h) {
          const int t = lane + 32 * h;
          if (((alive >> t) & 1ull) && key[h] > bk) {
            bk = key[h];
            bt = t;
          }
        }
        for (int o = 16; o; o >>= 1) {
          const long long ok = __shfl_xor_sync(FULL, bk, o);
          const int ot = __shfl_xor_sync(FULL, bt, o);
          if (ok > bk || (ok == bk && ot >= 0 && (bt < 0 || ot < bt))) {
            bk = ok;
            bt = ot;
          }
        }
        ++c;
        alive &= rows[bt];  // the candidates adjacent to the one added (not itself)
      }
      __syncwarp();  // the rows are rebuilt for the next seed
      p = 0;
    }
    while (p > 0) {
      // wide: the candidate of largest graph degree (ties: lowest rank), compared as one
      // 64-bit key
      long long bestkey = -1;
      int best = -1;
      for (int t = lane; t < p; t += 32) {
        const int32_t x = P[t];
        const int inner = 0;
        const int32_t d = min(__ldg(g.deg + __ldg(g.vert_of + x)), 0xFFFFF);
        const long long key = ((long long)inner << 40) | ((long long)d << 20) |
                              (long long)(0xFFFFF - (x & 0xFFFFF));
        if (key > bestkey) {
          bestkey = key;
          best = x;
        }
      }
      for (int o = 16; o; o >>= 1) {
        const long long ok = __shfl_xor_sync(FULL, bestkey, o);
        const int ob = __shfl_xor_sync(FULL, best, o);
        if (ok > bestkey || (ok == bestkey && ob >= 0 && (best < 0 || ob < best))) {
          bestkey = ok;
          best = ob;
        }
      }
      const int32_t u = best;
      ++c;
      // keep the candidates adjacent to u (in place: writes never pass the reads)
      int cnt = 0;
      for (int base = 0; base < p; base += 32) {
        const int t = base + lane;
        bool keep = false;
        int32_t x = 0;
        if (t < p) {
          x = P[t];
          if (x != u)
            keep = x > u ? contains64(g.oout, g.ooff[u], g.ooff[u + 1], x)
                         : contains64(g.oout, g.ooff[x], g.ooff[x + 1], u);
        }
        const unsigned bal = __ballot_sync(FULL, keep);
        __syncwarp();
        if (keep) P[cnt + __popc(bal & ((1u << lane) - 1))] = x;
        cnt += __popc(bal);
        __syncwarp();
      }
      p = cnt;
      if (c >= MAXD) break;
    }
    if (lane == 0) {
      const int st = subset_tau(c, k);
      if (st > 0) atomicMax(tau, st);
    }
    __syncwarp();
  }
}

// Warm start for seeds whose candidates all lie in the core bitmap (the dense core of the
// order, where near-cliques live): one warp per seed orders the candidates by their number of
// neighbours among the candidates (bitmap popcounts), then adds them greedily in that order
// when adjacent to every one added before, and publishes subset_tau of the clique's size.
// Like k_greedy_tau it records nothing (the answer is unchanged).  Seeds with more than
// kGreedyCoreMax candidates or outside the core are skipped.
constexpr int kGreedyCoreMax = 1024;
constexpr int kGreedyCoreWarps = 4;
__global__ void __launch_bounds__(kGreedyCoreWarps * 32)
    k_greedy_core_tau(DevGraph g, const int32_t* __restrict__ seeds, int64_t nseeds, int32_t k,
                      int32_t* __restrict__ tau) {
  __shared__ unsigned long long sP[kGreedyCoreWarps][64], sC[kGreedyCoreWarps][64];
  __shared__ unsigned long long sKey[kGreedyCoreWarps][kGreedyCoreMax];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const unsigned FULL = 0xffffffffu;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int cw = g.core_n >> 6;  // <= 64 words
  unsigned long long* P = sP[w];
  unsigned long long* C = sC[w];
  unsigned long long* key = sKey[w];
  for (int64_t it = warp; it < nseeds; it += nwarps) {
    const int32_t v = seeds[it];
    const int64_t b = g.ooff[v];
    const int p = (int)(g.ooff[v + 1] - b);
    if (p == 0 || p > kGreedyCoreMax || g.oout[b] < g.core_base) continue;
    for (int q = lane; q < 64; q += 32) {
      P[q] = 0ull;
      C[q] = 0ull;
    }
    __syncwarp();
    for (int t = lane; t < p; t += 32) {
      const int x = g.oout[b + t] - g.core_base;
      atomicOr(&P[x >> 6], 1ull << (x & 63));
    }
    __syncwarp();
    // key = (neighbours among the candidates) << 32 | (inverted core index: lower first)
    int n2 = 1;
    while (n2 < p) n2 <<= 1;
    for (int t = lane; t < n2; t += 32) {
      unsigned long long kk = 0ull;
      if (t < p) {
        const int x = g.oout[b + t] - g.core_base;
        const unsigned long long* row = g.core_bits + (int64_t)x * cw;
        int d = 0;
        for (int q = 0; q < cw; ++q) d += __popcll(__ldg(row + q) & P[q]);
        kk = ((unsigned long long)(d + 1) << 32) | (0xFFFFFFFFull - (unsigned)x);
      }
      key[t] = kk;
    }
    __syncwarp();
    // bitonic sort, descending
    for (int kk = 2; kk <= n2; kk <<= 1)
      for (int j = kk >> 1; j > 0; j >>= 1) {
        for (int i = lane; i < n2; i += 32) {
          const int l = i ^ j;
          if (l > i) {
            const unsigned long long a = key[i], c = key[l];
            const bool desc = (i & kk) == 0;
            if (desc ? (a < c) : (a > c)) {
              key[i] = c;
              key[l] = a;
            }
          }
        }
        __syncwarp();
      }
    // greedy: add each candidate, in that order, that is adjacent to every one added before
    int size = 1;
    for (int t = 0; t < p; ++t) {
      if ((t & 31) == 0) {  // cannot beat the current bound: stop (decided by lane 0)
        int stop = 0;
        if (lane == 0) stop = size + (p - t) <= ld_volatile(tau);
        if (__shfl_sync(FULL, stop, 0)) break;
      }
      const int x = (int)(0xFFFFFFFFull - (key[t] & 0xFFFFFFFFull));
      const unsigned long long* row = g.core_bits + (int64_t)x * cw;
      bool ok = true;
      for (int q = lane; q < cw; q += 32) ok &= (__ldg(row + q) & C[q]) == C[q];
      if (__all_sync(FULL, ok)) {
        if (lane == 0) C[x >> 6] |= 1ull << (x & 63);
        ++size;
      }
      __syncwarp();
    }
    if (lane == 0) {
      const int st = subset_tau(size, k);
      if (st > 0) atomicMax(tau, st);
    }
    __syncwarp();
  }
}

struct BucketPtrs {
  Rec* base[NB];
  int64_t fill[NB];  // current counts before the scatter
};

__global__ void k_stage_scatter(const Rec* stage, int64_t cnt, const BucketPtrs* __restrict__ bp,
                                int32_t* cursor) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < cnt;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (stage[i].nv <= 0) continue;
    int b = bucket_of(stage[i].bound);
    int64_t pos = bp->fill[b] + atomicAdd(&cursor[b], 1);
    bp->base[b][pos] = stage[i];
  }
}

__global__ void k_clear_stage(Rec* stage, int64_t cnt) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < cnt;
       i += (int64_t)gridDim.x * blockDim.x)
    stage[i].nv = 0;
}

// ---- final selection ----
__global__ void k_select(const Rec* res, int64_t cnt, int32_t tau, const DevGraph g,
                         int32_t* flag, int32_t* outV, int32_t* outN, int32_t* nsel) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < cnt;
       i += (int64_t)gridDim.x * blockDim.x) {
    int c = res[i].nv;
    if (c < tau || c > MAXD) continue;  // rows are cliques of 1..MAXD vertices
    int pos = atomicAdd(nsel, 1);
    int32_t ids[MAXD];
    for (int t = 0; t < c; ++t) ids[t] = __ldg(g.vert_of + res[i].V[t]);
    for (int a = 1; a < c; ++a) {  // insertion sort (c <= 32)
      int32_t x = ids[a];
      int b = a - 1;
      while (b >= 0 && ids[b] > x) {
        ids[b + 1] = ids[b];
        --b;
      }
      ids[b + 1] = x;
    }
    for (int t = 0; t < MAXD; ++t) outV[(int64_t)pos * MAXD + t] = t < c ? ids[t] : -1;
    outN[pos] = c;
  }
}

__global__ void k_gather_col(const int32_t* V, const int32_t* N, const int32_t* perm, int32_t n,
                             int col, uint32_t* key) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    int32_t r = perm[i];
    key[i] = col < 0 ? (uint32_t)(MAXD - N[r]) : (uint32_t)(V[(int64_t)r * MAXD + col] + 1);
  }
}

__global__ void k_iota(int32_t* a, int32_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    a[i] = (int32_t)i;
}

__global__ void k_emit(const int32_t* V, const int32_t* N, const int32_t* perm, int32_t count,
                       int32_t* outV, const int32_t* outOff, int64_t* outScore) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x) {
    int32_t r = perm[i];
    int c = N[r];
    outScore[i] = c;
    for (int t = 0; t < c; ++t) outV[outOff[i] + t] = V[(int64_t)r * MAXD + t];
  }
}

__global__ void k_sizes(const int32_t* N, const int32_t* perm, int32_t count, int32_t* sz) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x)
    sz[i] = N[perm[i]];
}

inline int grid_for(int64_t n) {
  int64_t b = (n + 255) / 256;
  return (int)std::max<int64_t>(1, std::min<int64_t>(b, 1 << 20));
}

// Device buffers of the dense-record search: one store per mask width and two task queues.
struct DenseBufs {
  DBuf<unsigned long long> rows2, rows4, rows8;
  DBuf<int32_t> vmap2, vmap4, vmap8, recV2, recV4, recV8, recN2, recN4, recN8, recP2, recP4,
      recP8;
  DBuf<unsigned long long> counters;  // [0] slots, [1] queue count, [2] next task, [3] ties
  DBuf<WTask> qa, qb;                 // task queues (wave input and output), grown on demand
  DBuf<WTask> qt;                     // tie nodes put back (all-cliques ranking)
  DBuf<unsigned long long> low2, low4, low8;  // tie-aware pruning masks per slot
  DBuf<int32_t> reclow2, reclow4, reclow8;
  DBuf<int32_t> lexbuf;                      // smallest id of each size-tau result
  DBuf<unsigned long long> lexcnt;
  DBuf<int32_t> cid2, cid4, cid8, rid2, rid4, rid8;  // full lexicographic bound, per slot
  DBuf<uint16_t> byid2, byid4, byid8;
  DBuf<int32_t> lexrows;                     // sorted id lists of the size-tau results
  DBuf<int32_t> lexL;                        // the list the bound compares with
  bool lex_allowed = false;  // all-cliques ranking, pruning on, ties not kept
  int64_t qcap = 0;          // current entries of each queue
  int64_t qmax = 0;          // entries a queue may grow to (NURI_TASK_QUEUE, default 16M)
  int32_t split_bits = 96;  // nodes with more candidates become tasks (measured best on B300)
};

// Entries each task queue may grow to (two queues): NURI_TASK_QUEUE, default 16M.
int64_t task_queue_max() {
  int64_t q = 1 << 24;
  if (const char* e = getenv("NURI_TASK_QUEUE")) q = std::max<int64_t>(16, atoll(e));
  return q;
}

// Device bytes of one store slot of the W-word tier (rows, vertex map, record, masks).
int64_t slot_bytes(int W) {
  const int64_t bmw = 64 * W;
  return bmw * W * 8 + bmw * 4 + MAXD * 4 + 8 + W * 8 + 4 + bmw * 6 + MAXD * 4;
}

// Store slots one dense pass uses at most: the records of a tier are searched in chunks of
// this many (a chunk's task waves finish before the next chunk reuses the slots).
int64_t slots_per_chunk(int W) {
  return std::max<int64_t>(64, kStoreBytes / slot_bytes(W));
}

WideStore make_store(DenseBufs& B, int W, int64_t nrec, cudaStream_t s) {
  const int64_t bmw = 64 * W;
  DBuf<unsigned long long>& rows = W == 2 ? B.rows2 : (W == 4 ? B.rows4 : B.rows8);
  DBuf<int32_t>& vmap = W == 2 ? B.vmap2 : (W == 4 ? B.vmap4 : B.vmap8);
  DBuf<int32_t>& recV = W == 2 ? B.recV2 : (W == 4 ? B.recV4 : B.recV8);
  DBuf<int32_t>& recN = W == 2 ? B.recN2 : (W == 4 ? B.recN4 : B.recN8);
  DBuf<int32_t>& recP = W == 2 ? B.recP2 : (W == 4 ? B.recP4 : B.recP8);
  DBuf<unsigned long long>& low = W == 2 ? B.low2 : (W == 4 ? B.low4 : B.low8);
  DBuf<int32_t>& reclow = W == 2 ? B.reclow2 : (W == 4 ? B.reclow4 : B.reclow8);
  DBuf<int32_t>& cid = W == 2 ? B.cid2 : (W == 4 ? B.cid4 : B.cid8);
  DBuf<int32_t>& rid = W == 2 ? B.rid2 : (W == 4 ? B.rid4 : B.rid8);
  DBuf<uint16_t>& byid = W == 2 ? B.byid2 : (W == 4 ? B.byid4 : B.byid8);
  if ((int64_t)recN.n < nrec) {
    int64_t cap = std::max<int64_t>(nrec, 256);
    rows.alloc(cap * bmw * W, s);
    vmap.alloc(cap * bmw, s);
    recV.alloc(cap * MAXD, s);
    recN.alloc(cap, s);
    recP.alloc(cap, s);
    if (B.lex_allowed) {
      low.alloc(cap * W, s);
      reclow.alloc(cap, s);
      cid.alloc(cap * bmw, s);
      byid.alloc(cap * bmw, s);
      rid.alloc(cap * MAXD, s);
    }
  }
  if (!B.counters.p) B.counters.alloc(4, s);
  if (B.lex_allowed && !B.qt.p) B.qt.alloc(kTieQueue, s);
  if (B.qmax == 0) {
    B.qmax = task_queue_max();
    if (const char* e = getenv("NURI_TASK_SPLIT")) B.split_bits = std::max(1, atoi(e));
  }
  // the record kernel queues up to one task per candidate of every record: start the queues
  // at that size (at least 1M entries); the task waves grow them further when they fill up
  const int64_t want = std::min<int64_t>(B.qmax, std::max<int64_t>(1 << 20, nrec * bmw));
  if (B.qcap < want) {
    B.qa.alloc(want, s);
    B.qb.alloc(want, s);
    B.qcap = want;
  }
  WideStore ws;
  ws.rows = rows.p;
  ws.vmap = vmap.p;
  ws.recV = recV.p;
  ws.recN = recN.p;
  ws.recP = recP.p;
  ws.nslots = B.counters.p;
  ws.slot_cap = nrec;
  ws.q_out = B.qa.p;
  ws.q_count = B.counters.p + 1;
  ws.q_cap = B.qcap;
  ws.split_bits = B.split_bits;
  ws.low = low.p;
  ws.reclow = reclow.p;
  ws.lex_tau = INT32_MIN;
  ws.lex_first = 0;
  ws.cid = B.lex_allowed ? cid.p : nullptr;
  ws.byid = B.lex_allowed ? byid.p : nullptr;
  ws.rid = B.lex_allowed ? rid.p : nullptr;
  ws.lexL = nullptr;
  ws.q_tie = B.lex_allowed ? B.qt.p : nullptr;
  ws.tie_count = B.counters.p + 3;
  ws.tie_cap = kTieQueue;
  return ws;
}

// Candidate results of size >= tau, copied from `in` to `out` (order not kept: the top-k merge
// sorts).  Rows below tau can never enter the top k, since tau only rises.
// With a tie list (lexL, for rows of size lex_tau): a row of that size whose sorted ids rank
// after lexL is dropped too (at least k known rows rank before it).  vert_of maps the row's
// ranks to ids.
__global__ void k_compact_results(const Rec* __restrict__ in, int64_t n, int32_t tau,
                                  Rec* __restrict__ out, unsigned long long* __restrict__ cnt,
                                  const int32_t* __restrict__ lexL, int32_t lex_tau,
                                  const int32_t* __restrict__ vert_of) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = warp; i < n; i += nwarps) {  // one warp per row
    const int nv = in[i].nv;
    if (nv < tau) continue;
    if (lexL && nv == lex_tau) {
      // the first position where the sorted row and lexL differ decides
      int first = INT32_MAX;
      bool after = false;
      for (int a = lane; a < nv; a += 32) {
        const int32_t x = __ldg(vert_of + in[i].V[a]);
        int r = 0;
        for (int b = 0; b < nv; ++b) r += __ldg(vert_of + in[i].V[b]) < x ? 1 : 0;
        if (x != lexL[r] && r < first) {
          first = r;
          after = x > lexL[r];
        }
      }
      int best = first;
      for (int o = 16; o; o >>= 1) best = min(best, __shfl_xor_sync(0xffffffffu, best, o));
      const bool drop = __any_sync(0xffffffffu, first == best && best != INT32_MAX && after);
      if (drop) continue;
    }
    unsigned long long slot = 0;
    if (lane == 0) slot = atomicAdd(cnt, 1ull);
    slot = __shfl_sync(0xffffffffu, slot, 0);
    Rec* o = out + slot;
    if (lane == 0) {
      o->nv = nv;
      o->bound = in[i].bound;
    }
    for (int a = lane; a < nv; a += 32) o->V[a] = in[i].V[a];
  }
}

// The device result set of one query pass.
struct ResultStore {
  DBuf<Rec> buf;
  int64_t cap = 0;
  DBuf<unsigned long long> cnt;
};

// Once the result set is half full, keep only its rows of size >= tau (into a buffer four
// times the rows kept, at least the current capacity), so that a long query does not
// overflow the set with cliques that tau has since passed.  A set that has already
// overflowed (rows lost) is left alone: the pass is then re-run with the final tau.
void compact_results(Ctx& cx, ResultStore& rs, cudaStream_t s, const int32_t* lexL = nullptr,
                     int32_t lex_tau = INT32_MIN) {
  // a caller's copy of the context may predate a compaction made further down: take the
  // current buffer first, whatever happens below
  cx.res = rs.buf.p;
  cx.res_cap = rs.cap;
  int64_t rc = 0;
  int32_t tau = 0;
  NURI_CUDA(cudaMemcpyAsync(&rc, &cx.st->res_count, 8, cudaMemcpyDeviceToHost, s));
  NURI_CUDA(cudaMemcpyAsync(&tau, &cx.st->tau, 4, cudaMemcpyDeviceToHost, s));
  NURI_CUDA(cudaStreamSynchronize(s));
  if (rc <= rs.cap / 2 || rc > rs.cap) return;
  if (!rs.cnt.p) rs.cnt.alloc(1, s);
  NURI_CUDA(cudaMemsetAsync(rs.cnt.p, 0, 8, s));
  DBuf<Rec> nb;
  nb.alloc(rs.cap, s);
  k_compact_results<<<std::max(1, std::min<int>((int)((rc + 7) / 8), sm_count() * 16)), 256, 0, s>>>(
      rs.buf.p, rc, tau, nb.p, rs.cnt.p, lexL, lex_tau, cx.g.vert_of);
  NURI_CUDA(cudaGetLastError());
  unsigned long long kept = 0;
  NURI_CUDA(cudaMemcpyAsync(&kept, rs.cnt.p, 8, cudaMemcpyDeviceToHost, s));
  NURI_CUDA(cudaStreamSynchronize(s));
  int64_t cap = rs.cap;
  if ((int64_t)kept * 4 > cap) {
    cap = (int64_t)kept * 4;
    DBuf<Rec> big;
    big.alloc(cap, s);
    if (kept)
      NURI_CUDA(cudaMemcpyAsync(big.p, nb.p, sizeof(Rec) * kept, cudaMemcpyDeviceToDevice, s));
    nb = std::move(big);
  }
  rs.buf = std::move(nb);
  rs.cap = cap;
  const int64_t kept64 = (int64_t)kept;
  NURI_CUDA(cudaMemcpyAsync(&cx.st->res_count, &kept64, 8, cudaMemcpyHostToDevice, s));
  NURI_CUDA(cudaStreamSynchronize(s));
  cx.res = rs.buf.p;
  cx.res_cap = rs.cap;
}

// Smallest original vertex id of every stored result of size tau (tie-aware pruning).
__global__ void k_row_minid(const Rec* __restrict__ res, int64_t n, int32_t tau,
                            const int32_t* __restrict__ vert_of, int32_t* __restrict__ out,
                            unsigned long long* __restrict__ cnt) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = warp; i < n; i += nwarps) {
    const int nv = res[i].nv;
    if (nv != tau) continue;
    int32_t m = INT32_MAX;
    for (int a = lane; a < nv; a += 32) m = min(m, __ldg(vert_of + res[i].V[a]));
    for (int o = 16; o; o >>= 1) m = min(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0) out[atomicAdd(cnt, 1ull)] = m;
  }
}

// The sorted original-id list of every stored result of size tau (tau ids each, rank by
// counting inside the row; one warp per row).
__global__ void k_rows_sorted(const Rec* __restrict__ res, int64_t n, int32_t tau,
                              const int32_t* __restrict__ vert_of, int32_t* __restrict__ out,
                              unsigned long long* __restrict__ cnt, int64_t cap) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = warp; i < n; i += nwarps) {
    if (res[i].nv != tau) continue;
    unsigned long long slot = 0;
    if (lane == 0) slot = atomicAdd(cnt, 1ull);
    slot = __shfl_sync(0xffffffffu, slot, 0);
    if ((int64_t)slot >= cap) continue;  // room for cap rows
    int32_t* o = out + (int64_t)slot * tau;
    for (int a = lane; a < tau; a += 32) {
      const int32_t x = __ldg(vert_of + res[i].V[a]);
      int r = 0;
      for (int b = 0; b < tau; ++b) r += __ldg(vert_of + res[i].V[b]) < x ? 1 : 0;
      o[r] = x;
    }
  }
}

// Per store slot: the candidates with vertex id <= first (mask of W words) and whether the
// record itself holds such a vertex.  One warp per slot.
template <int W>
__global__ void k_lex_low(WideStore ws, int64_t nslots, const int32_t* __restrict__ vert_of,
                          int32_t first, unsigned long long* __restrict__ low,
                          int32_t* __restrict__ reclow) {
  constexpr int BMW = 64 * W;
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t sl = warp; sl < nslots; sl += nwarps) {
    if (lane < W) low[sl * W + lane] = 0ull;
    __syncwarp();
    const int p = ws.recP[sl];
    for (int a = lane; a < p; a += 32)
      if (__ldg(vert_of + ws.vmap[sl * BMW + a]) <= first)
        atomicOr(&low[sl * W + (a >> 6)], 1ull << (a & 63));
    const int nv = ws.recN[sl];
    bool any_low = false;
    for (int a = lane; a < nv; a += 32) any_low |= __ldg(vert_of + ws.recV[sl * MAXD + a]) <= first;
    any_low = __any_sync(0xffffffffu, any_low);
    if (lane == 0) reclow[sl] = any_low ? 1 : 0;
    __syncwarp();
  }
}

// Device time and launches of the task kernel (CUDA events around every wave).
// Also the dense-record launches of the expansion kernel (rec_*: k_clique_expand<2/4/8>).
struct TailTime {
  double ms = 0.0;
  int64_t launches = 0;
  double rec_ms = 0.0;
  int64_t rec_launches = 0;
  cudaEvent_t a = nullptr, b = nullptr, c = nullptr, d = nullptr;
  TailTime() {
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    cudaEventCreate(&c);
    cudaEventCreate(&d);
  }
  ~TailTime() {
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaEventDestroy(c);
    cudaEventDestroy(d);
  }
};

// Tie-aware pruning threshold for the next wave: with c_hi known results larger than tau and
// at least need = k - c_hi stored results of size tau, lex_first = the need-th smallest of
// their smallest ids; every clique of size tau whose smallest id exceeds it ranks after k
// known results.  Off (lex_tau = INT32_MIN) when there are not enough such results yet.
template <int W>
void update_lex(const Ctx& cx, WideStore& ws, ResultStore& rs, DenseBufs& B, cudaStream_t s) {
  int32_t tau = 0;
  int64_t rc = 0;
  std::vector<int32_t> hist(MAXD + 2, 0);
  NURI_CUDA(cudaMemcpyAsync(&tau, &cx.st->tau, 4, cudaMemcpyDeviceToHost, s));
  NURI_CUDA(cudaMemcpyAsync(&rc, &cx.st->res_count, 8, cudaMemcpyDeviceToHost, s));
  NURI_CUDA(cudaMemcpyAsync(hist.data(), cx.st->hist, sizeof(int32_t) * (MAXD + 2),
                            cudaMemcpyDeviceToHost, s));
  NURI_CUDA(cudaStreamSynchronize(s));
  int64_t c_hi = 0;
  for (int c = std::max(tau + 1, 0); c <= MAXD + 1; ++c) c_hi += hist[c];
  const int64_t need = (int64_t)cx.k - c_hi;
  if (tau < 1 || tau > MAXD || need <= 0 || rc > rs.cap || rc <= 0) {
    ws.lex_tau = INT32_MIN;
    ws.lexL = nullptr;
    return;
  }
  if ((int64_t)B.lexbuf.n < rc) B.lexbuf.alloc(std::max<int64_t>(rc, 4096), s);
  if (!B.lexcnt.p) B.lexcnt.alloc(1, s);
  NURI_CUDA(cudaMemsetAsync(B.lexcnt.p, 0, 8, s));
  k_row_minid<<<std::max(1, std::min<int>((int)((rc + 7) / 8), sm_count() * 16)), 256, 0, s>>>(
      rs.buf.p, rc, tau, cx.g.vert_of, B.lexbuf.p, B.lexcnt.p);
  NURI_CUDA(cudaGetLastError());
  unsigned long long m = 0;
  NURI_CUDA(cudaMemcpyAsync(&m, B.lexcnt.p, 8, cudaMemcpyDeviceToHost, s));
  NURI_CUDA(cudaStreamSynchronize(s));
  if ((int64_t)m < need) {
    ws.lex_tau = INT32_MIN;
    ws.lexL = nullptr;
    return;
  }
  std::vector<int32_t> ids(m);
  NURI_CUDA(cudaMemcpyAsync(ids.data(), B.lexbuf.p, sizeof(int32_t) * m, cudaMemcpyDeviceToHost, s));
  NURI_CUDA(cudaStreamSynchronize(s));
  std::nth_element(ids.begin(), ids.begin() + (need - 1), ids.end());
  const int32_t first = ids[need - 1];
  // the full list: the need-th smallest sorted id list among (at most mcap of) the size-tau
  // results.  Taken over a subset it is no smaller than over all of them, and at least need
  // stored results are at or below it, so the bound stays valid (only weaker)
  if (ws.cid) {
    const int64_t mcap = std::min<int64_t>((int64_t)m, std::max<int64_t>(4096, 4 * need));
    if ((int64_t)B.lexrows.n < mcap * tau) B.lexrows.alloc(mcap * tau, s);
    NURI_CUDA(cudaMemsetAsync(B.lexcnt.p, 0, 8, s));
    k_rows_sorted<<<std::max(1, std::min<int>((int)((rc + 7) / 8), sm_count() * 16)), 256, 0, s>>>(
        rs.buf.p, rc, tau, cx.g.vert_of, B.lexrows.p, B.lexcnt.p, mcap);
    NURI_CUDA(cudaGetLastError());
    std::vector<int32_t> rows((size_t)mcap * tau);
    NURI_CUDA(cudaMemcpyAsync(rows.data(), B.lexrows.p, sizeof(int32_t) * mcap * tau,
                              cudaMemcpyDeviceToHost, s));
    NURI_CUDA(cudaStreamSynchronize(s));
    std::vector<int64_t> order(mcap);
    for (int64_t i = 0; i < mcap; ++i) order[i] = i;
    std::nth_element(order.begin(), order.begin() + (need - 1), order.end(),
                     [&](int64_t a, int64_t b) {
                       return std::lexicographical_compare(
                           rows.begin() + a * tau, rows.begin() + a * tau + tau,
                           rows.begin() + b * tau, rows.begin() + b * tau + tau);
                     });
    if ((int64_t)B.lexL.n < tau) B.lexL.alloc(MAXD, s);
    NURI_CUDA(cudaMemcpyAsync(B.lexL.p, rows.data() + order[need - 1] * tau,
                              sizeof(int32_t) * tau, cudaMemcpyHostToDevice, s));
    NURI_CUDA(cudaStreamSynchronize(s));
    ws.lexL = B.lexL.p;
  }
  if (ws.lex_tau == tau && ws.lex_first == first) return;  // masks still valid
  unsigned long long nslots = 0;
  NURI_CUDA(cudaMemcpyAsync(&nslots, B.counters.p, 8, cudaMemcpyDeviceToHost, s));
  NURI_CUDA(cudaStreamSynchronize(s));
  nslots = std::min<unsigned long long>(nslots, (unsigned long long)ws.slot_cap);
  if (nslots > 0) {
    k_lex_low<W><<<std::max(1, std::min<int>((int)((nslots + 7) / 8), sm_count() * 16)), 256, 0,
                   s>>>(ws, (int64_t)nslots, cx.g.vert_of, first,
                        const_cast<unsigned long long*>(ws.low), const_cast<int32_t*>(ws.reclow));
    NURI_CUDA(cudaGetLastError());
  }
  ws.lex_tau = tau;
  ws.lex_first = first;
}

// Dense records of one width: the warp kernel stores them and queues their children, then
// task waves run until the queue is empty.  A wave's grid is the resident capacity of the
// task kernel (lanes take tasks dynamically).  Records are taken in chunks of at most
// slots_per_chunk(W) so the store stays bounded; the queues grow (up to their maximum) when a
// wave's output passes an eighth of their size, the point where splitting would stop.
template <int W>
int64_t run_dense(Ctx cx, const Rec* recs, int64_t nrec, int grid, size_t dyn, DenseBufs& B,
                  TailTime& tt, ResultStore& rs, cudaStream_t s) {
  int64_t launched = 0;
  const bool trace = getenv("NURI_TRACE") != nullptr;
  static const int resident = [] {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_clique_tasks<W>, 128, 0) !=
            cudaSuccess ||
        per_sm < 1)
      per_sm = 4;
    return per_sm * sm_count();
  }();
  const int64_t chunk = slots_per_chunk(W);
  for (int64_t c0 = 0; c0 < nrec; c0 += chunk) {
    const int64_t cn = std::min<int64_t>(chunk, nrec - c0);
    WideStore ws = make_store(B, W, cn, s);
    NURI_CUDA(cudaMemsetAsync(B.counters.p, 0, 4 * sizeof(unsigned long long), s));
    NURI_CUDA(cudaMemsetAsync(&cx.st->work_next, 0, sizeof(int64_t), s));
    NURI_CUDA(cudaEventRecord(tt.c, s));
    k_clique_expand<W><<<grid, KCfg<W>::WARPS * 32, dyn, s>>>(cx, recs + c0, nullptr, cn, ws);
    NURI_CUDA(cudaGetLastError());
    NURI_CUDA(cudaEventRecord(tt.d, s));
    ++launched;
    bool in_is_a = true;  // the record kernel wrote its tasks to qa
    bool timed = false;   // a wave's events are pending
    bool rec_timed = true;
    while (true) {
      unsigned long long cnt = 0;
      NURI_CUDA(cudaMemcpyAsync(&cnt, B.counters.p + 1, 8, cudaMemcpyDeviceToHost, s));
      NURI_CUDA(cudaStreamSynchronize(s));
      if (rec_timed) {
        float ms = 0.f;
        NURI_CUDA(cudaEventElapsedTime(&ms, tt.c, tt.d));
        tt.rec_ms += ms;
        ++tt.rec_launches;
        rec_timed = false;
      }
      if (timed) {
        float ms = 0.f;
        NURI_CUDA(cudaEventElapsedTime(&ms, tt.a, tt.b));
        tt.ms += ms;
        ++tt.launches;
        timed = false;
      }
      int64_t n = std::min<int64_t>((int64_t)cnt, B.qcap);
      // the task queue is dry: one wave over the tie nodes put back (each is searched or, past
      // the threshold now, dropped; none is put back again)
      bool tie_wave = false;
      if (n == 0 && ws.q_tie) {
        unsigned long long nt = 0;
        NURI_CUDA(cudaMemcpyAsync(&nt, B.counters.p + 3, 8, cudaMemcpyDeviceToHost, s));
        NURI_CUDA(cudaStreamSynchronize(s));
        n = std::min<int64_t>((int64_t)nt, ws.tie_cap);
        tie_wave = n > 0;
      }
      if (n == 0) break;
      if (!tie_wave && n > B.qcap / 8 && B.qcap < B.qmax) {
        // grow both queues, keeping the pending tasks
        const int64_t cap = std::min<int64_t>(B.qmax, B.qcap * 4);
        DBuf<WTask> na, nb;
        na.alloc(cap, s);
        nb.alloc(cap, s);
        NURI_CUDA(cudaMemcpyAsync(na.p, in_is_a ? B.qa.p : B.qb.p, sizeof(WTask) * n,
                                  cudaMemcpyDeviceToDevice, s));
        B.qa = std::move(na);
        B.qb = std::move(nb);
        B.qcap = cap;
        ws.q_cap = cap;
        in_is_a = true;
      }
      compact_results(cx, rs, s, ws.lexL, ws.lex_tau);
      if (B.lex_allowed) update_lex<W>(cx, ws, rs, B, s);
      int32_t err = 0;
      NURI_CUDA(cudaMemcpyAsync(&err, &cx.st->err, 4, cudaMemcpyDeviceToHost, s));
      NURI_CUDA(cudaStreamSynchronize(s));
      if (err & 4) return launched;  // out of time: the caller reports it
      WTask* in = tie_wave ? B.qt.p : (in_is_a ? B.qa.p : B.qb.p);
      ws.q_out = in_is_a ? B.qb.p : B.qa.p;
      NURI_CUDA(cudaMemsetAsync(B.counters.p + 1, 0, (tie_wave ? 3 : 2) * sizeof(unsigned long long),
                                s));
      int tgrid = (int)std::min<int64_t>((n + 127) / 128, (int64_t)resident);
      ws.in_next = B.counters.p + 2;
      ws.in_n = n;
      WideStore wv = ws;
      if (tie_wave) wv.q_tie = nullptr;
      NURI_CUDA(cudaEventRecord(tt.a, s));
      k_clique_tasks<W><<<tgrid, 128, 0, s>>>(cx, wv, in, n, B.counters.p + 2);
      NURI_CUDA(cudaGetLastError());
      NURI_CUDA(cudaEventRecord(tt.b, s));
      timed = true;
      if (trace) {
        float ms = 0.f;
        NURI_CUDA(cudaEventSynchronize(tt.b));
        NURI_CUDA(cudaEventElapsedTime(&ms, tt.a, tt.b));
        unsigned long long exp = 0;
        int64_t nres = 0;
        NURI_CUDA(cudaMemcpy(&exp, &cx.st->expansions, 8, cudaMemcpyDeviceToHost));
        NURI_CUDA(cudaMemcpy(&nres, &cx.st->res_count, 8, cudaMemcpyDeviceToHost));
        fprintf(stderr,
                "[nuri]   dense W=%d wave %lld: %lld tasks (queue %lld), %.3f ms, nodes so far "
                "%llu, results %lld of %lld\n",
                W, (long long)launched, (long long)n, (long long)B.qcap, ms, exp,
                (long long)nres, (long long)rs.cap);
      }
      ++launched;
      in_is_a = !in_is_a;
    }
  }
  return launched;
}

// Narrow expansion over the batch, then the dense records it handed on (by mask width).
// ev0/ev1 bracket the CSR expansion launch alone; the task waves are timed in `tt`.
int64_t launch_expand(Ctx cx, const Rec* in, const int32_t* seeds, int64_t nin, int grid,
                      DBuf<Rec>& wide, DBuf<Rec>& mid, DBuf<Rec>& small, DenseBufs& B,
                      TailTime& tt, ResultStore& rs, cudaEvent_t ev0, cudaEvent_t ev1,
                      int64_t* tier_recs, cudaStream_t s) {
  const size_t dyn1 = sizeof(unsigned long long) * KCfg<1>::WARPS * 64;
  const size_t dyn2 = sizeof(unsigned long long) * KCfg<2>::WARPS * 64 * 2 * 2;
  const size_t dyn4 = sizeof(unsigned long long) * KCfg<4>::WARPS * 64 * 4 * 4;
  const size_t dynw = sizeof(unsigned long long) * KCfg<KWIDE>::WARPS * 64 * KWIDE * KWIDE;
  static const cudaError_t attr = cudaFuncSetAttribute(  // once per process (thread-safe init)
      k_clique_expand<KWIDE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dynw);
  static const cudaError_t attr4 = cudaFuncSetAttribute(
      k_clique_expand<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn4);
  NURI_CUDA(attr);
  NURI_CUDA(attr4);
  cx.wide = wide.p;
  cx.mid = mid.p;
  cx.small = small.p;
  NURI_CUDA(cudaEventRecord(ev0, s));
  WideStore none;
  memset(&none, 0, sizeof(none));
  k_clique_expand<1><<<grid, KCfg<1>::WARPS * 32, dyn1, s>>>(cx, in, seeds, nin, none);
  NURI_CUDA(cudaGetLastError());
  NURI_CUDA(cudaEventRecord(ev1, s));
  int64_t counts[3] = {0, 0, 0};  // wide_count, mid_count, small_count (adjacent fields)
  NURI_CUDA(cudaMemcpyAsync(counts, &cx.st->wide_count, 24, cudaMemcpyDeviceToHost, s));
  NURI_CUDA(cudaStreamSynchronize(s));
  int64_t launched = 1;
  tier_recs[0] += counts[2];
  tier_recs[1] += counts[1];
  tier_recs[2] += counts[0];
  if (counts[2] > 0) {
    compact_results(cx, rs, s);
    launched += run_dense<2>(cx, small.p, counts[2], grid, dyn2, B, tt, rs, s);
  }
  if (counts[1] > 0) {
    compact_results(cx, rs, s);
    launched += run_dense<4>(cx, mid.p, counts[1], grid, dyn4, B, tt, rs, s);
  }
  if (counts[0] > 0) {
    compact_results(cx, rs, s);
    launched += run_dense<KWIDE>(cx, wide.p, counts[0], grid * 2, dynw, B, tt, rs, s);
  }
  return launched;
}

struct HostBucket {
  DBuf<Rec> dev;            // device records [0, count)
  int64_t count = 0;
  std::vector<Rec*> spilled;          // pinned host chunks
  std::vector<int64_t> spilled_n;
  int64_t spilled_total = 0;
};

}  // namespace

// ---------------------------------------------------------------------------------------------
// Upper bound of the device memory one top-k clique query allocates on graph G (the buffers of
// topk_cliques below, at their bounded sizes): seeds and their sort, warm start, staging,
// frontier buckets up to frontier_cap records, round arrays, split-tier scratch, dense stores
// and task queues at their maximum, the initial result set twice (compaction) and the final
// merge.  A result set that outgrows its initial size adds to this (rare; the set is
// compacted to the rows >= tau first).
int64_t clique_query_bytes(const nuri_graph* G, int32_t k, uint32_t flags, int64_t frontier_cap) {
  const DevGraph& g = G->d;
  const bool no_prune = flags & NURI_NO_PRUNE;
  if (frontier_cap <= 0) frontier_cap = kDefaultFrontier;
  const int64_t rec = sizeof(Rec);
  const int64_t total_warps = (int64_t)sm_count() * 6 * KCfg<1>::WARPS;
  const int64_t n = std::max(g.n, 1);
  int64_t b = 0;
  b += 4 * n * 4 + 2 * n * 8 + 2 * NB * 4;                              // seeds, sort temp
  b += (int64_t)sm_count() * 4 * 8 * std::max(g.max_out, 1) * 4;       // warm start
  b += std::max<int64_t>(1 << 16, (int64_t)g.max_out * 8) * rec;        // staging
  if (g.max_out > PSMEM) b += total_warps * g.max_out * 4;              // P scratch
  if (g.max_out > 64 * KWIDE && !no_prune) b += total_warps * CB_ROWS * CB_W * 8;
  b += frontier_cap * rec + (int64_t)sizeof(BucketPtrs);                // frontier buckets
  b += 4 * kRoundRecs * rec + std::max<int64_t>(total_warps * 2, 4096) * rec;
  const int64_t res = std::max<int64_t>(1 << 16, (int64_t)k * 64);
  b += 2 * res * rec + res * (MAXD * 4 + 4 * 6 + 8);                   // results, merge
  if (g.max_out > 64) {                                                 // dense tiers
    for (int W : {2, 4, KWIDE}) b += slots_per_chunk(W) * slot_bytes(W);
    b += (2 * task_queue_max() + kTieQueue) * (int64_t)sizeof(WTask);
  }
  return b;
}

// Local memory the driver reserves, once per context, for the clique kernels: their largest
// per-thread frame times the threads the device can hold at once.
int64_t clique_local_reserve_bytes() {
  size_t frame = 0;
  auto take = [&](const void* f) {
    cudaFuncAttributes a;
    if (cudaFuncGetAttributes(&a, f) == cudaSuccess) frame = std::max(frame, a.localSizeBytes);
  };
  take((const void*)k_clique_tasks<2>);
  take((const void*)k_clique_tasks<4>);
  take((const void*)k_clique_tasks<KWIDE>);
  take((const void*)k_clique_expand<1>);
  take((const void*)k_clique_expand<2>);
  take((const void*)k_clique_expand<4>);
  take((const void*)k_clique_expand<KWIDE>);
  int dev = 0, threads = 2048;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&threads, cudaDevAttrMaxThreadsPerMultiProcessor, dev);
  return (int64_t)frame * sm_count() * threads;
}

void topk_cliques(nuri_graph* G, int32_t k, uint32_t flags, int64_t frontier_cap,
                  cudaStream_t s, nuri_result** out) {
  int64_t launches = 0;
  const DevGraph& g = G->d;
  DevTimer timer(s);
  const bool maximal = flags & NURI_CLIQUE_MAXIMAL;
  const bool no_prune = flags & NURI_NO_PRUNE;
  const bool keep_ties = flags & NURI_KEEP_TIES;
  if (frontier_cap <= 0) frontier_cap = kDefaultFrontier;
  const int n = g.n;

  const int grid = sm_count() * 6;  // CTAs of the narrow kernel: 6 x 4 warps per SM
  const int total_warps = grid * KCfg<1>::WARPS;
  const int64_t stage_cap = std::max<int64_t>(1 << 16, (int64_t)g.max_out * 8);

  DBuf<QState> st;
  st.alloc(1, s);
  std::atomic<int64_t> rounds_seen{0};  // read by the watchdog
  QueryWatchdog watchdog(st.p, &rounds_seen);
  DBuf<uint64_t> deadline;
  deadline.alloc(1, s);
  ++launches;
  k_set_deadline<<<1, 32, 0, s>>>(deadline.p, time_budget_ns());
  DBuf<int32_t> pscratch;
  if (g.max_out > PSMEM) pscratch.alloc((int64_t)total_warps * g.max_out, s);
  DBuf<unsigned long long> cbits;  // colouring check of split records (512 < |P| <= 1024)
  if (g.max_out > 64 * KWIDE && !no_prune)
    cbits.alloc((int64_t)total_warps * CB_ROWS * CB_W, s);
  DBuf<Rec> stage, deferred, inbuf, wide, mid, small;
  DenseBufs dense;
  if (G->clique_split_bits > 0) dense.split_bits = G->clique_split_bits;  // tuned per graph
  // tie-aware pruning: all-cliques ranking with pruning, exactly k rows (NURI_NO_LEX: off)
  dense.lex_allowed = !maximal && !no_prune && !keep_ties && getenv("NURI_NO_LEX") == nullptr;
  TailTime tail;
  stage.alloc(stage_cap, s);
  ++launches;
  k_clear_stage<<<grid_for(stage_cap), 256, 0, s>>>(stage.p, stage_cap);
  int64_t res_cap = std::max<int64_t>(1 << 16, (int64_t)k * 64);
  // initial result-buffer capacity override (exercises the overflow re-run in tests)
  if (const char* e = getenv("NURI_RESULT_CAP")) res_cap = std::max<int64_t>(1, atoll(e));
  int32_t tau_init = INT32_MIN;
  int restarts = 0;
  std::vector<HostBucket> buckets(NB);
  DBuf<BucketPtrs> bp_dev;  // the bucket table of a scatter (16 KB, passed through memory)

  // seeds: sorted by bound descending
  DBuf<int32_t> skeys, svals, skeys2, svals2, bhist;
  skeys.alloc(std::max(n, 1), s);
  svals.alloc(std::max(n, 1), s);
  skeys2.alloc(std::max(n, 1), s);
  svals2.alloc(std::max(n, 1), s);
  bhist.alloc(2 * NB, s);
  std::vector<int32_t> seed_hist(2 * NB, 0);
  if (n > 0) {
    ++launches;
    k_seed_bounds<<<grid_for(n), 256, 0, s>>>(g, G->part.index, G->part.count, skeys.p, svals.p);
    size_t tb = 0;
    cub::DeviceRadixSort::SortPairsDescending(nullptr, tb, skeys.p, skeys2.p, svals.p, svals2.p,
                                              n, 0, 32, s);
    DBuf<uint8_t> tmp;
    tmp.alloc(tb, s);
    NURI_CUDA(cub::DeviceRadixSort::SortPairsDescending(tmp.p, tb, skeys.p, skeys2.p, svals.p,
                                                        svals2.p, n, 0, 32, s));
    NURI_CUDA(cudaMemsetAsync(bhist.p, 0, sizeof(int32_t) * 2 * NB, s));
    ++launches;
    k_bucket_hist<<<grid_for(n), 256, 0, s>>>(skeys2.p, n, bhist.p);
    NURI_CUDA(cudaMemcpyAsync(seed_hist.data(), bhist.p, sizeof(int32_t) * 2 * NB,
                              cudaMemcpyDeviceToHost, s));
    NURI_CUDA(cudaStreamSynchronize(s));
  }
  // seed ranges per (class, bucket): class 1 first, then class 0, each by descending bound
  std::vector<int64_t> seed_lo(2 * NB), seed_hi(2 * NB);
  {
    int64_t pos = 0;
    for (int c = 1; c >= 0; --c)
      for (int b = NB - 1; b >= 0; --b) {
        seed_lo[c * NB + b] = pos;
        pos += seed_hist[c * NB + b];
        seed_hi[c * NB + b] = pos;
      }
  }

  // warm start: greedy cliques from the highest-bound seeds of each class lift tau before the
  // search (all-cliques ranking with pruning only)
  if (!maximal && !no_prune && n > 0 && k > 0) {
    DBuf<int32_t> gbuf, gtau;
    const int gblocks = sm_count() * 4;  // 8 warps each
    gbuf.alloc((int64_t)gblocks * 8 * std::max(g.max_out, 1), s);
    gtau.alloc(1, s);
    const int32_t neg = INT32_MIN;
    NURI_CUDA(cudaMemcpyAsync(gtau.p, &neg, 4, cudaMemcpyHostToDevice, s));
    const int64_t c0 = seed_lo[NB - 1], n0 = seed_lo[0] - c0;  // class 0 (wide) seeds
    const int64_t n1 = seed_hi[NB];                             // class 1 (narrow) seeds
    const int64_t take0 = std::min<int64_t>(n0, 4096), take1 = std::min<int64_t>(n1, 65536);
    if (take0 > 0) {
      ++launches;
      k_greedy_tau<<<gblocks, 256, 0, s>>>(g, svals2.p + c0, take0, k, gbuf.p, gtau.p);
    }
    if (take1 > 0) {
      ++launches;
      k_greedy_tau<<<gblocks, 256, 0, s>>>(g, svals2.p, take1, k, gbuf.p, gtau.p);
    }
    if (take0 > 0 && g.core_bits) {
      ++launches;
      k_greedy_core_tau<<<std::max<int64_t>(1, std::min<int64_t>((take0 + kGreedyCoreWarps - 1) /
                                                                      kGreedyCoreWarps,
                                                                  sm_count() * 8)),
                          kGreedyCoreWarps * 32, 0, s>>>(g, svals2.p + c0, take0, k, gtau.p);
    }
    NURI_CUDA(cudaGetLastError());
    int32_t gt = INT32_MIN;
    NURI_CUDA(cudaMemcpyAsync(&gt, gtau.p, 4, cudaMemcpyDeviceToHost, s));
    NURI_CUDA(cudaStreamSynchronize(s));
    tau_init = std::max(tau_init, gt);
  }

  QState hs;
  nuri_stats stats;
  memset(&stats, 0, sizeof(stats));
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

  ResultStore rs;
  while (true) {  // one pass; repeated only after a result-buffer overflow
    rs.buf.alloc(res_cap, s);
    rs.cap = res_cap;
    tail.ms = 0.0;
    tail.launches = 0;
    tail.rec_ms = 0.0;
    tail.rec_launches = 0;
    memset(&hs, 0, sizeof(hs));
    hs.tau = tau_init;
    NURI_CUDA(cudaMemcpyAsync(st.p, &hs, sizeof(hs), cudaMemcpyHostToDevice, s));
    for (auto& b : buckets) {
      b.count = 0;
      for (Rec* p : b.spilled) cudaFreeHost(p);
      b.spilled.clear();
      b.spilled_n.clear();
      b.spilled_total = 0;
    }
    // one cursor per seed class; a chunk may run across bound buckets.  Bucket 0 of class 0
    // holds only the seeds of other parts (bound 0) and is never taken.
    int64_t cls_next[2] = {seed_lo[NB - 1], seed_lo[NB + NB - 1]};
    const int64_t cls_end[2] = {seed_lo[0], seed_hi[NB]};
    auto bucket_at = [&](int c, int64_t pos) {
      for (int b = NB - 1; b >= 0; --b)
        if (pos < seed_hi[c * NB + b]) return b;
      return 0;
    };
    Ctx cx;
    cx.g = g;
    cx.st = st.p;
    cx.res = rs.buf.p;
    cx.res_cap = rs.cap;
    cx.stage = stage.p;
    cx.stage_cap = stage_cap;
    cx.pscratch = pscratch.p;
    cx.pscratch_stride = g.max_out;
    cx.cbits = cbits.p;
    cx.k = k;
    cx.maximal = maximal;
    cx.no_prune = no_prune;
    cx.deadline = deadline.p;
    cx.split_above = 64 * KWIDE;
    const bool trace = getenv("NURI_TRACE") != nullptr;  // per-round log on stderr
    // smaller split limit (exercises the frontier tier in tests)
    if (const char* e = getenv("NURI_SPLIT_ABOVE")) cx.split_above = std::max(1, atoi(e));
    int64_t rounds = 0;
    // per-round arrays of records handed to the dense tiers or sent back (at most kRoundRecs)
    auto ensure_round = [&](int64_t need) {
      need = std::max<int64_t>(need, 4096);
      if ((int64_t)deferred.n < need) deferred.alloc(need, s);
      if ((int64_t)wide.n < need) wide.alloc(need, s);
      if ((int64_t)mid.n < need) mid.alloc(need, s);
      if ((int64_t)small.n < need) small.alloc(need, s);
      cx.deferred = deferred.p;
    };
    // the first chunk is small: with tau still unset every node is a result, so a wide first
    // launch would fill the result set with small cliques; the chunk doubles every seed round
    // (once the warm start has set tau, results below it are not stored: start wide)
    int64_t seed_chunk = tau_init > 1 ? (1 << 16) : 512;

    while (true) {
      NURI_CUDA(cudaMemcpyAsync(&hs, st.p, sizeof(hs), cudaMemcpyDeviceToHost, s));
      NURI_CUDA(cudaStreamSynchronize(s));
      if (hs.err & 8)
        NURI_FAIL(NURI_ERR_CUDA,
                  "nuri_topk_cliques: internal error: frontier record %lld of round %lld is not "
                  "a clique record (nv %d)",
                  (long long)hs.bad_item, (long long)rounds, hs.bad_nv);
      if (hs.err & 1) NURI_FAIL(NURI_ERR_LIMIT, "nuri_topk_cliques: a clique exceeds %d vertices", MAXD);
      if (hs.err & 4)
        NURI_FAIL(NURI_ERR_TIMEOUT,
                  "nuri_topk_cliques: time budget exhausted after %lld rounds (%llu nodes "
                  "visited, tau %d)",
                  (long long)rounds, (unsigned long long)hs.expansions, hs.tau);
      compact_results(cx, rs, s);
      if (G->part.count > 1 && G->part.exchange) {
        // partitioned query: publish this part's threshold, prune with the best one known
        const int64_t loc = hs.tau == INT32_MIN ? INT64_MIN : (int64_t)hs.tau;
        const int64_t glob = G->part.exchange(G->part.ctx, 0, loc);
        if (glob > loc && glob <= MAXD + 1) {
          k_raise_tau<<<1, 32, 0, s>>>(&st.p->tau, (int32_t)glob);
          ++launches;
          NURI_CUDA(cudaGetLastError());
          hs.tau = (int32_t)glob;
        }
      }
      int32_t tau = hs.tau;
      // highest bucket with pending seeds (narrow class first) or frontier records
      int b_seed = -1, b_front = -1, seed_cls = -1;
      bool narrow_first = false;
      if (cls_next[1] < cls_end[1]) {
        int b = bucket_at(1, cls_next[1]);
        if (no_prune || b >= tau || b == NB - 1) {
          seed_cls = 1;
          b_seed = b;
          narrow_first = true;
        }
      }
      if (seed_cls < 0 && cls_next[0] < cls_end[0]) {
        seed_cls = 0;
        b_seed = bucket_at(0, cls_next[0]);
      }
      for (int b = NB - 1; b >= 0; --b)
        if (buckets[b].count + buckets[b].spilled_total > 0) {
          b_front = b;
          break;
        }
      int best = std::max(b_seed, b_front);
      if (best < 0) break;
      if (!no_prune && best < NB - 1 && best < tau) break;  // every remaining bound < tau
      if (narrow_first) b_front = -1;  // narrow seeds go before the frontier

      NURI_CUDA(cudaMemsetAsync(&st.p->work_next, 0, sizeof(int64_t), s));
      NURI_CUDA(cudaMemsetAsync(&st.p->stage_count, 0, sizeof(int64_t), s));
      NURI_CUDA(cudaMemsetAsync(&st.p->defer_count, 0, sizeof(int64_t), s));
      NURI_CUDA(cudaMemsetAsync(&st.p->wide_count, 0, 3 * sizeof(int64_t), s));
      int64_t nin = 0;
      int src_bucket = -1;
      if (b_front >= b_seed) {
        HostBucket& hb = buckets[b_front];
        src_bucket = b_front;
        if (hb.count == 0) {  // reload one spilled chunk
          Rec* hp = hb.spilled.back();
          int64_t hn = hb.spilled_n.back();
          hb.spilled.pop_back();
          hb.spilled_n.pop_back();
          hb.spilled_total -= hn;
          if ((int64_t)hb.dev.n < hn) hb.dev.alloc(hn, s);
          NURI_CUDA(cudaMemcpyAsync(hb.dev.p, hp, sizeof(Rec) * hn, cudaMemcpyHostToDevice, s));
          NURI_CUDA(cudaStreamSynchronize(s));
          cudaFreeHost(hp);
          hb.count = hn;
          stats.reloaded += hn;
        }
        const int64_t target = std::max<int64_t>(total_warps * 2, 4096);
        nin = std::min<int64_t>(hb.count, target);
        if ((int64_t)inbuf.n < target) inbuf.alloc(target, s);
        NURI_CUDA(cudaMemcpyAsync(inbuf.p, hb.dev.p + (hb.count - nin), sizeof(Rec) * nin,
                                  cudaMemcpyDeviceToDevice, s));
        hb.count -= nin;
        // a thin bucket does not fill a launch: take more records from the next buckets down
        // (still above tau and above the best pending seed); the order only changes the work
        for (int b2 = b_front - 1; b2 >= 0 && nin < target; --b2) {
          if (b2 < b_seed || (!no_prune && b2 < tau && b2 != NB - 1)) break;
          HostBucket& h2 = buckets[b2];
          if (h2.count == 0) continue;
          const int64_t take = std::min<int64_t>(h2.count, target - nin);
          NURI_CUDA(cudaMemcpyAsync(inbuf.p + nin, h2.dev.p + (h2.count - take),
                                    sizeof(Rec) * take, cudaMemcpyDeviceToDevice, s));
          h2.count -= take;
          nin += take;
        }
        ensure_round(nin);
        launches += launch_expand(cx, inbuf.p, nullptr, nin, grid, wide, mid, small, dense, tail, rs, ev0,
                                  ev1, stats.dense_records, s);
        cx.res = rs.buf.p;
        cx.res_cap = rs.cap;
      } else {
        const int c = seed_cls;
        int64_t lo = cls_next[c];
        int64_t hi = std::min<int64_t>(cls_end[c], lo + seed_chunk);
        // stop before seeds whose bound is already below tau, and (wide class) before
        // seeds that rank below the best frontier bucket
        if (!no_prune && tau > 0) hi = std::min(hi, seed_hi[c * NB + std::min(tau, NB - 1)]);
        if (!narrow_first && b_front >= 0) hi = std::min(hi, seed_hi[c * NB + b_front]);
        // narrow seeds (at most 64 candidates) never reach the dense tiers nor the split, so
        // their chunks are not bounded by the round arrays (unless a test lowers the split)
        const bool narrow_only = c == 1 && cx.split_above >= 64;
        if (!narrow_only) hi = std::min(hi, lo + kRoundRecs);
        hi = std::max(hi, std::min<int64_t>(lo + 1, cls_end[c]));
        nin = hi - lo;
        cls_next[c] = hi;
        seed_chunk = std::min<int64_t>(seed_chunk * 2, 1 << 20);
        ensure_round(narrow_only ? 0 : nin);
        launches += launch_expand(cx, nullptr, svals2.p + lo, nin, grid, wide, mid, small, dense, tail, rs,
                                  ev0, ev1, stats.dense_records, s);
        cx.res = rs.buf.p;
        cx.res_cap = rs.cap;
      }
      NURI_CUDA(cudaGetLastError());
      ++rounds;
      rounds_seen.fetch_add(1, std::memory_order_relaxed);
      if (trace) {
        float ms = 0.f;
        NURI_CUDA(cudaStreamSynchronize(s));
        NURI_CUDA(cudaEventElapsedTime(&ms, ev0, ev1));
        int64_t nwide = 0, nres = 0;
        int32_t tau_now = 0;
        NURI_CUDA(cudaMemcpy(&nwide, &st.p->wide_count, 8, cudaMemcpyDeviceToHost));
        NURI_CUDA(cudaMemcpy(&nres, &st.p->res_count, 8, cudaMemcpyDeviceToHost));
        NURI_CUDA(cudaMemcpy(&tau_now, &st.p->tau, 4, cudaMemcpyDeviceToHost));
        fprintf(stderr,
                "[nuri] round %lld %s bucket %d n %lld wide %lld tau %d -> %d, results %lld of "
                "%lld: %.3f ms\n",
                (long long)rounds, src_bucket >= 0 ? "frontier" : (narrow_first ? "narrow" : "seeds"),
                b_front >= b_seed ? b_front : b_seed, (long long)nin, (long long)nwide, tau,
                tau_now, (long long)nres, (long long)rs.cap, ms);
      }
      // staging (children) and deferred parents -> buckets, by bound
      int64_t scnt = 0, dcnt = 0;
      NURI_CUDA(cudaMemcpyAsync(&scnt, &st.p->stage_count, 8, cudaMemcpyDeviceToHost, s));
      NURI_CUDA(cudaMemcpyAsync(&dcnt, &st.p->defer_count, 8, cudaMemcpyDeviceToHost, s));
      NURI_CUDA(cudaStreamSynchronize(s));
      {
        float ms = 0.f;
        NURI_CUDA(cudaEventElapsedTime(&ms, ev0, ev1));
        stats.expand_ms += ms;
        stats.expand_launches += 1;
      }
      scnt = std::min(scnt, stage_cap);
      auto scatter = [&](Rec* arr, int64_t cnt) {
        if (cnt <= 0) return;
        std::vector<int32_t> sh(NB, 0);
        NURI_CUDA(cudaMemsetAsync(bhist.p, 0, sizeof(int32_t) * NB, s));
        ++launches;
        k_stage_hist<<<grid_for(cnt), 256, 0, s>>>(arr, cnt, bhist.p);
        NURI_CUDA(cudaMemcpyAsync(sh.data(), bhist.p, sizeof(int32_t) * NB,
                                  cudaMemcpyDeviceToHost, s));
        NURI_CUDA(cudaStreamSynchronize(s));
        BucketPtrs bp;
        for (int b = 0; b < NB; ++b) {
          HostBucket& hb = buckets[b];
          int64_t need = hb.count + sh[b];
          if (need > (int64_t)hb.dev.n) {
            DBuf<Rec> nb;
            nb.alloc(std::max<int64_t>(need * 2, 1024), s);
            if (hb.count)
              NURI_CUDA(cudaMemcpyAsync(nb.p, hb.dev.p, sizeof(Rec) * hb.count,
                                        cudaMemcpyDeviceToDevice, s));
            hb.dev = std::move(nb);
          }
          bp.base[b] = hb.dev.p;
          bp.fill[b] = hb.count;
        }
        NURI_CUDA(cudaMemsetAsync(bhist.p, 0, sizeof(int32_t) * NB, s));
        ++launches;
        if (!bp_dev.p) bp_dev.alloc(1, s);
        NURI_CUDA(cudaMemcpyAsync(bp_dev.p, &bp, sizeof(BucketPtrs), cudaMemcpyHostToDevice, s));
        k_stage_scatter<<<grid_for(cnt), 256, 0, s>>>(arr, cnt, bp_dev.p, bhist.p);
        ++launches;
        k_clear_stage<<<grid_for(cnt), 256, 0, s>>>(arr, cnt);
        for (int b = 0; b < NB; ++b) buckets[b].count += sh[b];
      };
      scatter(stage.p, scnt);
      scatter(deferred.p, dcnt);
      (void)src_bucket;
      // spill the lowest buckets while the device frontier is above its capacity
      int64_t total = 0;
      for (auto& hb : buckets) total += hb.count;
      for (int b = 0; b < NB && total > frontier_cap; ++b) {
        HostBucket& hb = buckets[b];
        if (hb.count == 0) continue;
        if (!no_prune && b < tau && b < NB - 1) {  // dominated: drop instead of spilling
          total -= hb.count;
          stats.pruned += hb.count;
          hb.count = 0;
          continue;
        }
        Rec* hp = nullptr;
        if (cudaMallocHost((void**)&hp, sizeof(Rec) * hb.count) != cudaSuccess)
          NURI_FAIL(NURI_ERR_OOM, "nuri_topk_cliques: pinned host allocation failed");
        NURI_CUDA(cudaMemcpyAsync(hp, hb.dev.p, sizeof(Rec) * hb.count, cudaMemcpyDeviceToHost, s));
        hb.spilled.push_back(hp);
        hb.spilled_n.push_back(hb.count);
        hb.spilled_total += hb.count;
        stats.spilled += hb.count;
        total -= hb.count;
        hb.count = 0;
      }
      NURI_CUDA(cudaStreamSynchronize(s));
    }
    // the state read at the top of the last round predates that round's result compaction
    // (which lowers res_count): read it again before the rows are selected
    NURI_CUDA(cudaMemcpyAsync(&hs, st.p, sizeof(hs), cudaMemcpyDeviceToHost, s));
    NURI_CUDA(cudaStreamSynchronize(s));
    // drop what is left (every remaining bound < tau)
    for (auto& b : buckets) {
      for (Rec* p : b.spilled) cudaFreeHost(p);
      b.spilled.clear();
      b.spilled_n.clear();
      b.spilled_total = 0;
      b.count = 0;
    }
    stats.rounds += rounds;
    if (hs.res_count > rs.cap) {
      // every result with size >= tau_final was counted: re-run with that threshold and room
      int64_t need = 0;
      for (int c = std::max(hs.tau, 0); c <= MAXD; ++c) need += hs.hist[c];
      res_cap = std::max<int64_t>(need + 1024, rs.cap);
      tau_init = hs.tau;
      ++restarts;
      continue;
    }
    break;
  }

  // ---- top-k merge: rows with size >= tau, ordered by (size desc, ids lex asc) ----
  int64_t cnt = hs.res_count;
  int32_t tau = hs.tau;
  DBuf<int32_t> selV, selN, nsel, flag;
  selV.alloc(std::max<int64_t>(cnt, 1) * MAXD, s);
  selN.alloc(std::max<int64_t>(cnt, 1), s);
  nsel.alloc(1, s);
  flag.alloc(1, s);
  NURI_CUDA(cudaMemsetAsync(nsel.p, 0, 4, s));
  if (cnt > 0) { ++launches; k_select<<<grid_for(cnt), 256, 0, s>>>(rs.buf.p, cnt, tau, g, flag.p, selV.p, selN.p, nsel.p); }
  int32_t ns = 0;
  NURI_CUDA(cudaMemcpyAsync(&ns, nsel.p, 4, cudaMemcpyDeviceToHost, s));
  NURI_CUDA(cudaStreamSynchronize(s));
  int maxc = 0;
  for (int c = MAXD; c >= 1; --c)
    if (hs.hist[c] > 0) {
      maxc = c;
      break;
    }
  DBuf<int32_t> perm, perm2;
  DBuf<uint32_t> key, key2;
  perm.alloc(std::max(ns, 1), s);
  perm2.alloc(std::max(ns, 1), s);
  key.alloc(std::max(ns, 1), s);
  key2.alloc(std::max(ns, 1), s);
  if (ns > 0) {
    ++launches;
    k_iota<<<grid_for(ns), 256, 0, s>>>(perm.p, ns);
    size_t tb = 0;
    cub::DeviceRadixSort::SortPairs(nullptr, tb, key.p, key2.p, perm.p, perm2.p, ns, 0, 32, s);
    DBuf<uint8_t> tmp;
    tmp.alloc(tb, s);
    // least significant column first; the size key last (stable passes)
    for (int col = maxc - 1; col >= -1; --col) {
      ++launches;
      k_gather_col<<<grid_for(ns), 256, 0, s>>>(selV.p, selN.p, perm.p, ns, col, key.p);
      NURI_CUDA(cub::DeviceRadixSort::SortPairs(tmp.p, tb, key.p, key2.p, perm.p, perm2.p, ns,
                                                0, 32, s));
      std::swap(perm.p, perm2.p);
    }
  }
  int32_t count = ns;
  if (!keep_ties) count = std::min(count, k);
  // row sizes on the host for the offsets
  std::vector<int32_t> sizes(count);
  DBuf<int32_t> dsz;
  dsz.alloc(std::max(count, 1), s);
  if (count > 0) {
    ++launches;
    k_sizes<<<grid_for(count), 256, 0, s>>>(selN.p, perm.p, count, dsz.p);
    NURI_CUDA(cudaMemcpyAsync(sizes.data(), dsz.p, sizeof(int32_t) * count, cudaMemcpyDeviceToHost, s));
    NURI_CUDA(cudaStreamSynchronize(s));
  }
  int64_t nverts = 0;
  for (int i = 0; i < count; ++i) nverts += sizes[i];
  nuri_result* r = new_result(0, count, nverts, 0, false);
  r->vert_off[0] = 0;
  for (int i = 0; i < count; ++i) r->vert_off[i + 1] = r->vert_off[i] + sizes[i];
  r->edge_off[0] = 0;
  for (int i = 0; i < count; ++i) r->edge_off[i + 1] = 0;
  if (count > 0) {
    DBuf<int32_t> dOff, dV;
    DBuf<int64_t> dS;
    dOff.alloc(count + 1, s);
    dV.alloc(std::max<int64_t>(nverts, 1), s);
    dS.alloc(count, s);
    NURI_CUDA(cudaMemcpyAsync(dOff.p, r->vert_off, sizeof(int32_t) * (count + 1),
                              cudaMemcpyHostToDevice, s));
    ++launches;
    k_emit<<<grid_for(count), 256, 0, s>>>(selV.p, selN.p, perm.p, count, dV.p, dOff.p, dS.p);
    NURI_CUDA(cudaMemcpyAsync(r->verts, dV.p, sizeof(int32_t) * nverts, cudaMemcpyDeviceToHost, s));
    NURI_CUDA(cudaMemcpyAsync(r->score, dS.p, sizeof(int64_t) * count, cudaMemcpyDeviceToHost, s));
    NURI_CUDA(cudaStreamSynchronize(s));
  }
  stats.expansions += (int64_t)hs.expansions;
  stats.pruned += (int64_t)hs.pruned;
  stats.dequeued += (int64_t)hs.dequeued;
  stats.adj_bytes += (int64_t)hs.adj_bytes;
  stats.tail_words = (int64_t)hs.tail_words;
  stats.expand_ms += tail.rec_ms;  // the dense-record launches of the expansion kernel
  stats.expand_launches += tail.rec_launches;
  stats.lex_pruned = (int64_t)hs.lex_pruned;
  stats.tail_ms = tail.ms;
  stats.tail_launches = tail.launches;
  stats.results_stored = hs.res_count;
  stats.threshold = hs.tau == INT32_MIN ? INT64_MIN : hs.tau;
  stats.restarts = restarts;
  stats.device_ms = timer.stop();
  stats.launches = launches;
  r->stats = stats;
  *out = r;
}

}  // namespace nuri
