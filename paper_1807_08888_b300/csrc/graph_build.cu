// Device graph construction: the engine loads the data graph into memory (Section 5) and runs
// each vertex's index initialize() at load time (Section 4.3, Listing 3).
//
// Steps (all on the device, stream-ordered):
//   1. validate ids, expand each input pair to both directions, drop self-loops
//   2. radix-sort the 64-bit (row, col) keys, drop duplicates -> undirected CSR (sorted rows)
//   3. degeneracy orientation for cliques: rank = position in the batch-peeling order (core
//      decomposition); out-rows in rank space keep only neighbours of larger rank, so every
//      out-row has at most degeneracy(G) entries
//   4. label segments: each row grouped by neighbour label, each group sorted by score desc
//   5. hop/label max index, H rounds of a gather-max over neighbours
#include <cub/cub.cuh>

#include <mutex>

#include "nuri_internal.cuh"

namespace nuri {
namespace {

constexpr int kThreads = 256;

inline int blocks_for(int64_t n, int threads = kThreads) {
  int64_t b = (n + threads - 1) / threads;
  if (b < 1) b = 1;
  if (b > (1ll << 30)) b = 1ll << 30;
  return (int)b;
}

inline int bitlen(uint64_t x) {
  int b = 0;
  while (x) {
    ++b;
    x >>= 1;
  }
  return b;
}

__global__ void k_validate(const int32_t* __restrict__ src, const int32_t* __restrict__ dst,
                           int64_t m, int32_t n, int32_t* bad) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m;
       i += (int64_t)gridDim.x * blockDim.x) {
    int32_t a = src[i], b = dst[i];
    if (a < 0 || a >= n || b < 0 || b >= n) atomicExch(bad, 1);
  }
}

// both directions of every pair; a self-loop becomes the sentinel row n
__global__ void k_expand_pairs(const int32_t* __restrict__ src, const int32_t* __restrict__ dst,
                               int64_t m, int32_t n, uint64_t* __restrict__ keys) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m;
       i += (int64_t)gridDim.x * blockDim.x) {
    uint32_t a = (uint32_t)src[i], b = (uint32_t)dst[i];
    uint64_t sent = (uint64_t)(uint32_t)n << 32;
    keys[2 * i] = a == b ? sent : ((uint64_t)a << 32) | b;
    keys[2 * i + 1] = a == b ? sent : ((uint64_t)b << 32) | a;
  }
}

__global__ void k_split_keys(const uint64_t* __restrict__ keys, int64_t nnz,
                             int32_t* __restrict__ adj, int32_t* __restrict__ deg) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nnz;
       i += (int64_t)gridDim.x * blockDim.x) {
    uint64_t k = keys[i];
    adj[i] = (int32_t)(uint32_t)k;
    atomicAdd(&deg[(uint32_t)(k >> 32)], 1);
  }
}

__global__ void k_rank_keys(const int32_t* __restrict__ deg, int32_t n,
                            uint64_t* __restrict__ keys) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    keys[i] = ((uint64_t)(uint32_t)deg[i] << 32) | (uint32_t)i;
}

__global__ void k_rank_split(const uint64_t* __restrict__ keys, int32_t n,
                             int32_t* __restrict__ vert_of, int32_t* __restrict__ rank_of) {
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n;
       r += (int64_t)gridDim.x * blockDim.x) {
    int32_t v = (int32_t)(uint32_t)keys[r];
    vert_of[r] = v;
    rank_of[v] = (int32_t)r;
  }
}

// ---- degeneracy order by batch peeling -------------------------------------------------
// A vertex is removed in the first batch where its remaining degree is <= k (k = the current
// core level); at that moment at most k of its neighbours remain, so every vertex has at most
// degeneracy(G) neighbours later in the (batch, id) order.
__global__ void k_peel_init(const int32_t* __restrict__ deg, int32_t n, int32_t* __restrict__ rem,
                            int32_t* __restrict__ batch) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x) {
    rem[v] = deg[v];
    batch[v] = -1;
  }
}

__global__ void k_peel_min(const int32_t* __restrict__ rem, const int32_t* __restrict__ batch,
                           int32_t n, int32_t* out) {
  int32_t best = INT32_MAX;
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x)
    if (batch[v] < 0) best = min(best, rem[v]);
  for (int o = 16; o; o >>= 1) best = min(best, __shfl_xor_sync(0xffffffffu, best, o));
  if ((threadIdx.x & 31) == 0) atomicMin(out, best);
}

__global__ void k_peel_select(const int32_t* __restrict__ rem, int32_t* __restrict__ batch,
                              int32_t n, int32_t k, int32_t b, int32_t* __restrict__ front,
                              int32_t* cnt) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x)
    if (batch[v] < 0 && rem[v] <= k) {
      batch[v] = b;
      front[atomicAdd(cnt, 1)] = (int32_t)v;
    }
}

__global__ void k_peel_remove(const int64_t* __restrict__ off, const int32_t* __restrict__ adj,
                              const int32_t* __restrict__ front, int32_t nfront, int32_t k,
                              int32_t b, int32_t* __restrict__ rem, int32_t* __restrict__ batch,
                              int32_t* __restrict__ next, int32_t* ncnt) {
  // one warp per removed vertex
  const int lane = threadIdx.x & 31;
  for (int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; w < nfront;
       w += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    int32_t v = front[w];
    for (int64_t t = off[v] + lane; t < off[v + 1]; t += 32) {
      int32_t u = adj[t];
      if (*(volatile int32_t*)(batch + u) >= 0) continue;
      int32_t old = atomicSub(rem + u, 1);
      if (old - 1 <= k && atomicCAS(batch + u, -1, b + 1) == -1) next[atomicAdd(ncnt, 1)] = u;
    }
  }
}

// The rest of the peel in one CTA, once at most kTailVertices vertices are left (the long
// tail of small batches would otherwise cost a launch and a host round trip each).  Same rule
// as the batch loop on the host: when the front is empty, k rises to the smallest remaining
// degree and every unassigned vertex with remaining degree <= k forms batch b; removing a
// batch lowers its neighbours' degrees and those that drop to <= k form batch b + 1.
//
// The tail runs on a local copy of the subgraph it still touches, so that every step of a
// batch is a shared-memory atomic instead of a chain of global ones:
//   local ids [0, nf) are the current front (assigned, not yet removed), [nf, nl) the
//   unassigned vertices; gid maps a local id to its vertex, loc the other way (-1 outside);
//   the local row of i (loff/ladj, 16-bit local ids) lists i's unassigned neighbours.
// Shared memory holds each local vertex's remaining degree as a 16-bit half of a 32-bit word
// (a degree never passes nl - 1 <= 65535 in a simple graph, and never goes below zero, so
// the halves never borrow from each other) and one assigned bit per local vertex.
constexpr int32_t kTailVertices = 1 << 16;
constexpr int64_t kHeavyRow = 512;  // rows longer than this are walked by the whole CTA
constexpr int kHeavyList = 256;     // heavy rows per batch handled that way (the rest by warps)

__global__ void k_tail_ids(const int32_t* __restrict__ batch, int32_t n,
                           const int32_t* __restrict__ front, int32_t nf, int32_t nl,
                           int32_t* __restrict__ gid, int32_t* __restrict__ loc, int32_t* cnt) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x) {
    if (v < nf) {
      gid[v] = front[v];
      loc[front[v]] = (int32_t)v;
    }
    if (batch[v] < 0) {
      const int32_t i = nf + atomicAdd(cnt, 1);
      if (i < nl) {  // the host checks the count before using the ids
        gid[i] = (int32_t)v;
        loc[v] = i;
      }
    }
  }
}

// one warp per local vertex: the number of its unassigned neighbours
__global__ void k_tail_count(const int64_t* __restrict__ off, const int32_t* __restrict__ adj,
                             const int32_t* __restrict__ gid, const int32_t* __restrict__ loc,
                             int32_t nl, int32_t nf, int64_t* __restrict__ lcnt) {
  const int lane = threadIdx.x & 31;
  for (int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; i < nl;
       i += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    const int32_t v = gid[i];
    int32_t c = 0;
    for (int64_t t = off[v] + lane; t < off[v + 1]; t += 32) c += loc[adj[t]] >= nf;
    for (int o = 16; o; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if (lane == 0) lcnt[i] = c;
  }
}

__global__ void k_tail_fill(const int64_t* __restrict__ off, const int32_t* __restrict__ adj,
                            const int32_t* __restrict__ gid, const int32_t* __restrict__ loc,
                            int32_t nl, int32_t nf, const int64_t* __restrict__ loff,
                            uint16_t* __restrict__ ladj) {
  const int lane = threadIdx.x & 31;
  for (int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; i < nl;
       i += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    const int32_t v = gid[i];
    int64_t pos = loff[i];
    for (int64_t t0 = off[v]; t0 < off[v + 1]; t0 += 32) {
      const int64_t t = t0 + lane;
      const int32_t u = t < off[v + 1] ? loc[adj[t]] : -1;
      const bool keep = u >= nf;
      const unsigned m = __ballot_sync(0xffffffffu, keep);
      if (keep) ladj[pos + __popc(m & ((1u << lane) - 1))] = (uint16_t)u;
      pos += __popc(m);
    }
  }
}

// out[0] = the largest k reached; out[1] = 0 on success, 1 if a front came out empty while
// vertices remained, 2 if a remaining degree did not fit 16 bits (neither can happen; both
// reported instead of looping or miscounting).
__global__ void __launch_bounds__(1024) k_peel_tail(
    const int64_t* __restrict__ loff, const uint16_t* __restrict__ ladj,
    const int32_t* __restrict__ gid, const int32_t* __restrict__ rem, int32_t nl, int32_t nf0,
    int32_t k0, int32_t b0, int32_t* __restrict__ batch, int32_t* fa, int32_t* fb,
    int32_t* out) {
  extern __shared__ uint32_t s_dyn[];
  uint32_t* s_rem = s_dyn;                    // (nl + 1) / 2 words, two 16-bit degrees each
  uint32_t* s_done = s_dyn + (nl + 1) / 2;    // (nl + 31) / 32 words, one assigned bit each
  __shared__ int32_t s_nfront, s_nnext, s_k, s_min, s_nheavy, s_bad;
  __shared__ int32_t s_heavy[kHeavyList];
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5, nwarps = nthr >> 5;
  const int32_t nwords = (nl + 31) / 32;
  if (tid == 0) s_bad = 0;
  __syncthreads();
  for (int32_t w = tid; w < (nl + 1) / 2; w += nthr) {
    uint32_t lo = 0, hi = 0;
    const int32_t i = 2 * w;
    if (i >= nf0) lo = (uint32_t)rem[gid[i]];
    if (i + 1 < nl && i + 1 >= nf0) hi = (uint32_t)rem[gid[i + 1]];
    if ((lo | hi) > 0xffffu) atomicExch(&s_bad, 1);
    s_rem[w] = (lo & 0xffffu) | (hi << 16);
  }
  for (int32_t w = tid; w < nwords; w += nthr) {
    uint32_t bits = 0;  // the front is assigned; bits past nl stay set so scans skip them
    for (int j = 0; j < 32; ++j) {
      const int32_t i = w * 32 + j;
      if (i < nf0 || i >= nl) bits |= 1u << j;
    }
    s_done[w] = bits;
  }
  for (int32_t i = tid; i < nf0; i += nthr) fa[i] = i;
  if (tid == 0) {
    s_nfront = nf0;
    s_nnext = 0;
    s_k = k0;
    s_nheavy = 0;
  }
  __syncthreads();
  if (s_bad) {
    if (tid == 0) out[1] = 2;
    return;
  }
  int32_t* front = fa;
  int32_t* next = fb;
  int32_t b = b0;
  int32_t remaining = nl;
  auto rem_of = [&](int32_t i) -> int32_t { return (s_rem[i >> 1] >> ((i & 1) * 16)) & 0xffffu; };
  while (remaining > 0) {
    if (s_nfront == 0) {
      // k rises to the smallest remaining degree; every unassigned vertex at or below it
      // forms batch b
      if (tid == 0) s_min = INT32_MAX;
      __syncthreads();
      int32_t mn = INT32_MAX;
      for (int32_t w = tid; w < nwords; w += nthr) {
        uint32_t open = ~s_done[w];
        while (open) {
          const int j = __ffs(open) - 1;
          open &= open - 1;
          mn = min(mn, rem_of(w * 32 + j));
        }
      }
      for (int o = 16; o; o >>= 1) mn = min(mn, __shfl_xor_sync(0xffffffffu, mn, o));
      if (lane == 0) atomicMin(&s_min, mn);
      __syncthreads();
      if (tid == 0) s_k = max(s_k, s_min);
      __syncthreads();
      const int32_t k = s_k;
      for (int32_t w = tid; w < nwords; w += nthr) {
        uint32_t open = ~s_done[w], take = 0;
        while (open) {
          const int j = __ffs(open) - 1;
          open &= open - 1;
          if (rem_of(w * 32 + j) <= k) take |= 1u << j;
        }
        if (take) {
          s_done[w] |= take;  // one thread owns each word here
          const int c = __popc(take);
          int32_t at = atomicAdd(&s_nfront, c);
          while (take) {
            const int j = __ffs(take) - 1;
            take &= take - 1;
            const int32_t i = w * 32 + j;
            front[at++] = i;
            batch[gid[i]] = b;
          }
        }
      }
      __syncthreads();
      if (s_nfront == 0) {
        if (tid == 0) out[1] = 1;
        return;
      }
    }
    const int32_t k = s_k, nf = s_nfront;
    // light front vertices: one warp each; heavy ones (long rows): the whole CTA, one at a
    // time, so that a hub's row is not walked by one warp's chain of atomics
    auto drop = [&](int32_t u) {
      const uint32_t bit = 1u << (u & 31);
      if (s_done[u >> 5] & bit) return;
      const int sh = (u & 1) * 16;
      const int32_t old = (int32_t)((atomicSub(&s_rem[u >> 1], 1u << sh) >> sh) & 0xffffu);
      if (old - 1 <= k && !(atomicOr(&s_done[u >> 5], bit) & bit)) {
        next[atomicAdd(&s_nnext, 1)] = u;
        batch[gid[u]] = b + 1;
      }
    };
    for (int w = warp; w < nf; w += nwarps) {
      const int32_t v = front[w];
      const int64_t lo = loff[v], hi = loff[v + 1];
      if (hi - lo > kHeavyRow) {
        int slot = -1;
        if (lane == 0) slot = atomicAdd(&s_nheavy, 1);
        slot = __shfl_sync(0xffffffffu, slot, 0);
        if (slot < kHeavyList) {
          if (lane == 0) s_heavy[slot] = v;
          continue;
        }
      }
      // four loads in flight per lane before the atomics that use them
      for (int64_t t = lo + lane; t < hi; t += 128) {
        int32_t u[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) u[q] = t + 32 * q < hi ? (int32_t)ladj[t + 32 * q] : -1;
#pragma unroll
        for (int q = 0; q < 4; ++q)
          if (u[q] >= 0) drop(u[q]);
      }
    }
    __syncthreads();
    const int nh = min(s_nheavy, kHeavyList);
    for (int h = 0; h < nh; ++h) {
      const int32_t v = s_heavy[h];
      for (int64_t t = loff[v] + tid; t < loff[v + 1]; t += nthr) drop(ladj[t]);
    }
    __syncthreads();
    {
      int32_t* t = front;
      front = next;
      next = t;
    }
    remaining -= nf;
    ++b;
    if (tid == 0) {
      s_nheavy = 0;
      s_nfront = s_nnext;
      s_nnext = 0;
    }
    __syncthreads();
  }
  if (tid == 0) {
    out[0] = s_k;
    out[1] = 0;
  }
}

__global__ void k_peel_keys(const int32_t* __restrict__ batch, int32_t n,
                            uint64_t* __restrict__ keys) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x)
    keys[v] = ((uint64_t)(uint32_t)batch[v] << 32) | (uint32_t)v;
}

// one key per directed entry whose target has the larger rank; the rest become sentinels
__global__ void k_orient_keys(const uint64_t* __restrict__ ckeys, int64_t nnz,
                              const int32_t* __restrict__ rank_of, int32_t n,
                              uint64_t* __restrict__ okeys) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nnz;
       i += (int64_t)gridDim.x * blockDim.x) {
    uint64_t k = ckeys[i];
    int32_t rv = rank_of[(uint32_t)(k >> 32)], ru = rank_of[(uint32_t)k];
    okeys[i] = rv < ru ? (((uint64_t)(uint32_t)rv << 32) | (uint32_t)ru)
                       : ((uint64_t)(uint32_t)n << 32);
  }
}

__global__ void k_orient_split(const uint64_t* __restrict__ okeys, int64_t cnt,
                               int32_t* __restrict__ oout, int32_t* __restrict__ odeg) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < cnt;
       i += (int64_t)gridDim.x * blockDim.x) {
    uint64_t k = okeys[i];
    oout[i] = (int32_t)(uint32_t)k;
    atomicAdd(&odeg[(uint32_t)(k >> 32)], 1);
  }
}

__global__ void k_max_i32(const int32_t* __restrict__ a, int64_t n, int32_t* out) {
  int32_t best = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    best = max(best, a[i]);
  for (int o = 16; o; o >>= 1) best = max(best, __shfl_xor_sync(0xffffffffu, best, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, best);
}

__global__ void k_max_u8(const uint8_t* __restrict__ a, int64_t n, int32_t* out) {
  int32_t best = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    best = max(best, (int32_t)a[i]);
  for (int o = 16; o; o >>= 1) best = max(best, __shfl_xor_sync(0xffffffffu, best, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, best);
}

__global__ void k_min_i32(const int32_t* __restrict__ a, int64_t n, int32_t* out) {
  int32_t best = INT32_MAX;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    best = min(best, a[i]);
  for (int o = 16; o; o >>= 1) best = min(best, __shfl_xor_sync(0xffffffffu, best, o));
  if ((threadIdx.x & 31) == 0) atomicMin(out, best);
}

// label segments: secondary key (score desc, id asc), value = (row << 32 | col)
__global__ void k_seg_keys(const uint64_t* __restrict__ ckeys, int64_t nnz,
                           const int32_t* __restrict__ score, uint64_t* __restrict__ skey,
                           uint64_t* __restrict__ sval) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nnz;
       i += (int64_t)gridDim.x * blockDim.x) {
    uint64_t k = ckeys[i];
    uint32_t u = (uint32_t)k;
    uint32_t inv = (uint32_t)(INT32_MAX - score[u]);  // score >= 0 -> larger score first
    skey[i] = ((uint64_t)inv << 32) | u;
    sval[i] = k;
  }
}

__global__ void k_seg_primary(const uint64_t* __restrict__ sval, int64_t nnz,
                              const uint8_t* __restrict__ labels, int32_t L,
                              uint64_t* __restrict__ pkey) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nnz;
       i += (int64_t)gridDim.x * blockDim.x) {
    uint64_t k = sval[i];
    uint32_t v = (uint32_t)(k >> 32), u = (uint32_t)k;
    pkey[i] = (uint64_t)v * (uint64_t)L + labels[u];
  }
}

__global__ void k_seg_fill(const uint64_t* __restrict__ pkey, const uint64_t* __restrict__ sval,
                           int64_t nnz, const int32_t* __restrict__ score,
                           int2* __restrict__ seg, int32_t* __restrict__ segcnt) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nnz;
       i += (int64_t)gridDim.x * blockDim.x) {
    uint32_t u = (uint32_t)sval[i];
    seg[i] = make_int2((int32_t)u, score[u]);
    atomicAdd(&segcnt[pkey[i]], 1);
  }
}

__global__ void k_i32_to_i64(const int32_t* __restrict__ a, int64_t n, int64_t* __restrict__ b) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    b[i] = a[i];
}

__global__ void k_label_keys(const uint8_t* __restrict__ labels, int32_t n,
                             uint64_t* __restrict__ keys) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    keys[i] = ((uint64_t)labels[i] << 32) | (uint32_t)i;
}

__global__ void k_label_split(const uint64_t* __restrict__ keys, int32_t n,
                              int32_t* __restrict__ vert, int32_t* __restrict__ cnt) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    vert[i] = (int32_t)(uint32_t)keys[i];
    atomicAdd(&cnt[keys[i] >> 32], 1);
  }
}

__global__ void k_gmax(const uint8_t* __restrict__ labels, const int32_t* __restrict__ score,
                       int32_t n, int32_t* __restrict__ gmax) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    atomicMax(&gmax[labels[i]], score[i]);
}

}  // namespace

// ---------------------------------------------------------------------------------------------
// Hop/label max index (Section 4.3, Listing 3), cumulative-hop reading:
//   idx_h(v)[l] = max over x in N(v) of max(own(x)[l], idx_{h-1}(x)[l]),
//   own(x)[l] = score(x) if label(x) == l else -1, idx_0 = -1.
// i.e. the max score of a label-l vertex reachable from v by a walk of 1..h edges.
// One warp per vertex: lanes are split into 32/L groups that take different neighbours, each
// lane of a group owns one label, and the groups are reduced with shuffles.  Vertices with
// degree above kHeavy get a whole CTA (one warp per neighbour slice + shared reduction).
// HBM traffic per round: the CSR row (4 B per entry) plus the L-vector of each neighbour
// (4*L B per entry, gathered), plus the output row.
// ---------------------------------------------------------------------------------------------
namespace {

constexpr int kHeavy = 2048;

template <int LP>
__global__ void __launch_bounds__(256) k_hop_round_light(
    const int64_t* __restrict__ off, const int32_t* __restrict__ adj,
    const uint8_t* __restrict__ labels, const int32_t* __restrict__ score,
    const int32_t* __restrict__ prev, int32_t n, int32_t L, int32_t* __restrict__ cur) {
  constexpr int G = 32 / LP;  // neighbours per step
  const int lane = threadIdx.x & 31;
  const int grp = lane / LP, l = lane % LP;
  const bool active = l < L;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t v = warp; v < n; v += nwarps) {
    int64_t b = off[v], e = off[v + 1];
    if (e - b > kHeavy) continue;  // handled by the CTA kernel
    int32_t acc = -1;
    if (active)
      for (int64_t i = b + grp; i < e; i += G) {
        int32_t x = __ldg(adj + i);
        int32_t own = (__ldg(labels + x) == l) ? __ldg(score + x) : -1;
        int32_t p = prev ? __ldg(prev + (int64_t)x * L + l) : -1;
        acc = max(acc, max(own, p));
      }
#pragma unroll
    for (int o = LP; o < 32; o <<= 1) acc = max(acc, __shfl_xor_sync(0xffffffffu, acc, o));
    if (grp == 0 && active) cur[(int64_t)v * L + l] = acc;
  }
}

template <int LP>
__global__ void __launch_bounds__(512) k_hop_round_heavy(
    const int64_t* __restrict__ off, const int32_t* __restrict__ adj,
    const uint8_t* __restrict__ labels, const int32_t* __restrict__ score,
    const int32_t* __restrict__ prev, const int32_t* __restrict__ heavy, int32_t nheavy,
    int32_t L, int32_t* __restrict__ cur) {
  constexpr int G = 32 / LP;
  __shared__ int32_t red[16][32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int grp = lane / LP, l = lane % LP;
  const bool active = l < L;
  for (int32_t hi = blockIdx.x; hi < nheavy; hi += gridDim.x) {
    int32_t v = heavy[hi];
    int64_t b = off[v], e = off[v + 1];
    int32_t acc = -1;
    if (active)
      for (int64_t i = b + (int64_t)w * G + grp; i < e; i += (int64_t)nw * G) {
        int32_t x = __ldg(adj + i);
        int32_t own = (__ldg(labels + x) == l) ? __ldg(score + x) : -1;
        int32_t p = prev ? __ldg(prev + (int64_t)x * L + l) : -1;
        acc = max(acc, max(own, p));
      }
#pragma unroll
    for (int o = LP; o < 32; o <<= 1) acc = max(acc, __shfl_xor_sync(0xffffffffu, acc, o));
    red[w][lane] = acc;
    __syncthreads();
    if (w == 0) {
      int32_t a = red[0][lane];
      for (int j = 1; j < nw; ++j) a = max(a, red[j][lane]);
      if (lane < L && lane < LP) cur[(int64_t)v * L + lane] = a;
    }
    __syncthreads();
  }
}

// general L (any label count): one thread per (v, l) pair, serial over the row
__global__ void k_hop_round_generic(const int64_t* __restrict__ off,
                                    const int32_t* __restrict__ adj,
                                    const uint8_t* __restrict__ labels,
                                    const int32_t* __restrict__ score,
                                    const int32_t* __restrict__ prev, int32_t n, int32_t L,
                                    int32_t* __restrict__ cur) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < (int64_t)n * L;
       t += (int64_t)gridDim.x * blockDim.x) {
    int64_t v = t / L;
    int l = (int)(t % L);
    int32_t acc = -1;
    for (int64_t i = off[v]; i < off[v + 1]; ++i) {
      int32_t x = adj[i];
      int32_t own = labels[x] == l ? score[x] : -1;
      int32_t p = prev ? prev[(int64_t)x * L + l] : -1;
      acc = max(acc, max(own, p));
    }
    cur[t] = acc;
  }
}

__global__ void k_collect_heavy(const int64_t* __restrict__ off, int32_t n,
                                int32_t* __restrict__ heavy, int32_t* __restrict__ cnt) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x)
    if (off[v + 1] - off[v] > kHeavy) heavy[atomicAdd(cnt, 1)] = (int32_t)v;
}

template <int LP>
void hop_rounds_t(const DevGraph& d, const int32_t* score, int32_t H, int32_t* idx,
                  const int32_t* heavy, int32_t nheavy, cudaStream_t s) {
  int grid = sm_count() * 8;
  for (int h = 1; h <= H; ++h) {
    const int32_t* prev = h == 1 ? nullptr : idx + (int64_t)(h - 2) * d.n * d.L;
    int32_t* cur = idx + (int64_t)(h - 1) * d.n * d.L;
    k_hop_round_light<LP><<<grid, 256, 0, s>>>(d.off, d.adj, d.labels, score, prev, d.n, d.L,
                                               cur);
    if (nheavy)
      k_hop_round_heavy<LP><<<std::min(nheavy, sm_count() * 4), 512, 0, s>>>(
          d.off, d.adj, d.labels, score, prev, heavy, nheavy, d.L, cur);
  }
}

}  // namespace

void build_hop_index(const DevGraph& d, const int32_t* score, int32_t H, int32_t* idx,
                     cudaStream_t s) {
  if (H <= 0 || d.n == 0) return;
  DBuf<int32_t> heavy, cnt;
  heavy.alloc(d.n, s);
  cnt.alloc(1, s);
  NURI_CUDA(cudaMemsetAsync(cnt.p, 0, 4, s));
  k_collect_heavy<<<blocks_for(d.n), kThreads, 0, s>>>(d.off, d.n, heavy.p, cnt.p);
  int32_t nheavy = 0;
  NURI_CUDA(cudaMemcpyAsync(&nheavy, cnt.p, 4, cudaMemcpyDeviceToHost, s));
  NURI_CUDA(cudaStreamSynchronize(s));
  if (d.L <= 1) hop_rounds_t<1>(d, score, H, idx, heavy.p, nheavy, s);
  else if (d.L <= 2) hop_rounds_t<2>(d, score, H, idx, heavy.p, nheavy, s);
  else if (d.L <= 4) hop_rounds_t<4>(d, score, H, idx, heavy.p, nheavy, s);
  else if (d.L <= 8) hop_rounds_t<8>(d, score, H, idx, heavy.p, nheavy, s);
  else if (d.L <= 16) hop_rounds_t<16>(d, score, H, idx, heavy.p, nheavy, s);
  else if (d.L <= 32) hop_rounds_t<32>(d, score, H, idx, heavy.p, nheavy, s);
  else
    for (int h = 1; h <= H; ++h) {
      const int32_t* prev = h == 1 ? nullptr : idx + (int64_t)(h - 2) * d.n * d.L;
      k_hop_round_generic<<<sm_count() * 8, 256, 0, s>>>(d.off, d.adj, d.labels, score, prev,
                                                         d.n, d.L,
                                                         idx + (int64_t)(h - 1) * d.n * d.L);
    }
  NURI_CUDA(cudaGetLastError());
}

// weight-ranked (or degree-ranked) label segments
void build_label_segments(const DevGraph& d, const uint64_t* ckeys, const int32_t* score,
                          DBuf<int2>& seg, DBuf<int64_t>* lsoff, cudaStream_t s) {
  const int64_t nnz = d.nnz;
  DBuf<uint64_t> k1, v1, k2, v2;
  k1.alloc(nnz, s);
  v1.alloc(nnz, s);
  k2.alloc(nnz, s);
  v2.alloc(nnz, s);
  k_seg_keys<<<blocks_for(nnz), kThreads, 0, s>>>(ckeys, nnz, score, k1.p, v1.p);
  size_t tmp_bytes = 0;
  cub::DeviceRadixSort::SortPairs(nullptr, tmp_bytes, k1.p, k2.p, v1.p, v2.p, nnz, 0, 64, s);
  DBuf<uint8_t> tmp;
  tmp.alloc(tmp_bytes, s);
  NURI_CUDA(cub::DeviceRadixSort::SortPairs(tmp.p, tmp_bytes, k1.p, k2.p, v1.p, v2.p, nnz, 0,
                                            64, s));
  // v2 now in (score desc, id asc) order; stable sort by (row, label)
  k_seg_primary<<<blocks_for(nnz), kThreads, 0, s>>>(v2.p, nnz, d.labels, d.L, k1.p);
  int end_bit = bitlen((uint64_t)d.n * (uint64_t)d.L + 1);
  size_t tmp2 = 0;
  cub::DeviceRadixSort::SortPairs(nullptr, tmp2, k1.p, k2.p, v2.p, v1.p, nnz, 0, end_bit, s);
  if (tmp2 > tmp_bytes) {
    tmp.alloc(tmp2, s);
    tmp_bytes = tmp2;
  }
  NURI_CUDA(cub::DeviceRadixSort::SortPairs(tmp.p, tmp_bytes, k1.p, k2.p, v2.p, v1.p, nnz, 0,
                                            end_bit, s));
  seg.alloc(nnz, s);
  if (lsoff) {
    int64_t nl = (int64_t)d.n * d.L;
    DBuf<int32_t> cnt;
    cnt.alloc(nl + 1, s);
    NURI_CUDA(cudaMemsetAsync(cnt.p, 0, sizeof(int32_t) * (nl + 1), s));
    k_seg_fill<<<blocks_for(nnz), kThreads, 0, s>>>(k2.p, v1.p, nnz, score, seg.p, cnt.p);
    DBuf<int64_t> cnt64;
    cnt64.alloc(nl + 1, s);
    k_i32_to_i64<<<blocks_for(nl + 1), kThreads, 0, s>>>(cnt.p, nl + 1, cnt64.p);
    lsoff->alloc(nl + 1, s);
    size_t t3 = 0;
    cub::DeviceScan::ExclusiveSum(nullptr, t3, cnt64.p, lsoff->p, nl + 1, s);
    DBuf<uint8_t> tmp3;
    tmp3.alloc(t3, s);
    NURI_CUDA(cub::DeviceScan::ExclusiveSum(tmp3.p, t3, cnt64.p, lsoff->p, nl + 1, s));
  } else {
    DBuf<int32_t> dummy;
    dummy.alloc((int64_t)d.n * d.L + 1, s);
    NURI_CUDA(cudaMemsetAsync(dummy.p, 0, dummy.bytes(), s));
    k_seg_fill<<<blocks_for(nnz), kThreads, 0, s>>>(k2.p, v1.p, nnz, score, seg.p, dummy.p);
  }
  NURI_CUDA(cudaGetLastError());
}

// Degeneracy (batch-peeling) order keys (batch << 32 | id); false if the peel needs more than
// kMaxPeelBatches batches (then the caller uses the degree order).
static bool peel_order(nuri_graph* g, uint64_t* keys, cudaStream_t s) {
  constexpr int kMaxPeelBatches = 20000;
  const int32_t n = g->d.n;
  DBuf<int32_t> rem, batch, fa, fb, cnt;
  rem.alloc(n, s);
  batch.alloc(n, s);
  fa.alloc(n, s);
  fb.alloc(n, s);
  cnt.alloc(2, s);
  k_peel_init<<<blocks_for(n), kThreads, 0, s>>>(g->deg.p, n, rem.p, batch.p);
  int64_t remaining = n;
  int32_t k = 0, b = 0, nfront = 0;
  int32_t* front = fa.p;
  int32_t* next = fb.p;
  int32_t maxk = 0;
  while (remaining > 0) {
    if (b > kMaxPeelBatches) return false;
    if (remaining <= kTailVertices) {
      // finish on the device in one CTA, on the local subgraph of what is left
      const int32_t nl = (int32_t)remaining;
      DBuf<int32_t> gid, loc, tout;
      DBuf<int64_t> lcnt, loff;
      gid.alloc(nl, s);
      loc.alloc(n, s);
      lcnt.alloc(nl + 1, s);
      loff.alloc(nl + 1, s);
      tout.alloc(2, s);
      NURI_CUDA(cudaMemsetAsync(loc.p, 0xff, sizeof(int32_t) * (size_t)n, s));
      NURI_CUDA(cudaMemsetAsync(cnt.p, 0, 4, s));
      k_tail_ids<<<blocks_for(n), kThreads, 0, s>>>(batch.p, n, front, nfront, nl, gid.p, loc.p,
                                                    cnt.p);
      NURI_CUDA(cudaMemsetAsync(lcnt.p + nl, 0, sizeof(int64_t), s));
      const int wgrid = (int)std::min<int64_t>((nl + 7) / 8, sm_count() * 16);
      k_tail_count<<<wgrid, 256, 0, s>>>(g->off.p, g->adj.p, gid.p, loc.p, nl, nfront, lcnt.p);
      size_t tb = 0;
      cub::DeviceScan::ExclusiveSum(nullptr, tb, lcnt.p, loff.p, nl + 1, s);
      DBuf<uint8_t> tmp;
      tmp.alloc(tb, s);
      NURI_CUDA(cub::DeviceScan::ExclusiveSum(tmp.p, tb, lcnt.p, loff.p, nl + 1, s));
      int32_t nu = 0;
      int64_t lnnz = 0;
      NURI_CUDA(cudaMemcpyAsync(&nu, cnt.p, 4, cudaMemcpyDeviceToHost, s));
      NURI_CUDA(cudaMemcpyAsync(&lnnz, loff.p + nl, 8, cudaMemcpyDeviceToHost, s));
      NURI_CUDA(cudaStreamSynchronize(s));
      if ((int64_t)nu + nfront != nl) return false;  // the count kept on the host is off
      DBuf<uint16_t> ladj;
      ladj.alloc(std::max<int64_t>(lnnz, 1), s);
      k_tail_fill<<<wgrid, 256, 0, s>>>(g->off.p, g->adj.p, gid.p, loc.p, nl, nfront, loff.p,
                                        ladj.p);
      const size_t smem = sizeof(uint32_t) * (size_t)((nl + 1) / 2 + (nl + 31) / 32);
      NURI_CUDA(cudaFuncSetAttribute(k_peel_tail, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem));
      // fronts hold local ids; fa/fb have room for n >= nl entries
      k_peel_tail<<<1, 1024, smem, s>>>(loff.p, ladj.p, gid.p, rem.p, nl, nfront, k, b,
                                        batch.p, front, next, tout.p);
      NURI_CUDA(cudaGetLastError());
      int32_t to[2] = {0, 1};
      NURI_CUDA(cudaMemcpyAsync(to, tout.p, 8, cudaMemcpyDeviceToHost, s));
      NURI_CUDA(cudaStreamSynchronize(s));
      if (to[1] != 0) return false;
      maxk = std::max(maxk, to[0]);
      remaining = 0;
      break;
    }
    if (nfront == 0) {
      int32_t init = INT32_MAX;
      NURI_CUDA(cudaMemcpyAsync(cnt.p, &init, 4, cudaMemcpyHostToDevice, s));
      k_peel_min<<<blocks_for(n), kThreads, 0, s>>>(rem.p, batch.p, n, cnt.p);
      int32_t mn = 0;
      NURI_CUDA(cudaMemcpyAsync(&mn, cnt.p, 4, cudaMemcpyDeviceToHost, s));
      NURI_CUDA(cudaStreamSynchronize(s));
      k = std::max(k, mn);
      NURI_CUDA(cudaMemsetAsync(cnt.p, 0, 4, s));
      k_peel_select<<<blocks_for(n), kThreads, 0, s>>>(rem.p, batch.p, n, k, b, front, cnt.p);
      NURI_CUDA(cudaMemcpyAsync(&nfront, cnt.p, 4, cudaMemcpyDeviceToHost, s));
      NURI_CUDA(cudaStreamSynchronize(s));
      if (nfront == 0) return false;  // cannot happen while vertices remain
    }
    maxk = std::max(maxk, k);
    NURI_CUDA(cudaMemsetAsync(cnt.p + 1, 0, 4, s));
    k_peel_remove<<<std::min<int64_t>((nfront + 7) / 8, sm_count() * 16), 256, 0, s>>>(
        g->off.p, g->adj.p, front, nfront, k, b, rem.p, batch.p, next, cnt.p + 1);
    remaining -= nfront;
    int32_t nn = 0;
    NURI_CUDA(cudaMemcpyAsync(&nn, cnt.p + 1, 4, cudaMemcpyDeviceToHost, s));
    NURI_CUDA(cudaStreamSynchronize(s));
    std::swap(front, next);
    nfront = nn;
    ++b;
  }
  g->degeneracy = maxk;
  k_peel_keys<<<blocks_for(n), kThreads, 0, s>>>(batch.p, n, keys);
  return true;
}

// The core bitmap: one warp per core rank r scans r's out-row (ranks above r, all in the
// core) and sets both directions of every edge.
constexpr int32_t kCoreRanks = 4096;
__global__ void k_core_bits(const int64_t* __restrict__ ooff, const int32_t* __restrict__ oout,
                            int32_t base, int32_t cn, unsigned long long* __restrict__ bits) {
  const int lane = threadIdx.x & 31;
  const int32_t words = cn / 64;
  for (int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; w < cn;
       w += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    const int32_t r = base + (int32_t)w;
    for (int64_t t = ooff[r] + lane; t < ooff[r + 1]; t += 32) {
      const int32_t x = oout[t] - base;
      atomicOr(&bits[w * words + (x >> 6)], 1ull << (x & 63));
      atomicOr(&bits[(int64_t)x * words + (w >> 6)], 1ull << (w & 63));
    }
  }
}

// ---- edge weights (ranking isomorphism matches by cumulative edge weight) -------------------
namespace {

// Position of b in the id-sorted row of a, or -1.
__device__ __forceinline__ int64_t row_find(const int64_t* __restrict__ off,
                                            const int32_t* __restrict__ adj, int32_t a,
                                            int32_t b) {
  int64_t lo = off[a], hi = off[a + 1];
  const int64_t end = hi;
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (__ldg(adj + mid) < b) lo = mid + 1;
    else hi = mid;
  }
  return lo < end && __ldg(adj + lo) == b ? lo : -1;
}

// Every pair (a, b), a != b, raises both directions of its edge to at least w; flag[0]: an id
// outside [0, n), flag[1]: a negative weight, flag[2]: a pair that is not an edge.
__global__ void k_ew_scatter(const int64_t* __restrict__ off, const int32_t* __restrict__ adj,
                             int32_t n, const int32_t* __restrict__ src,
                             const int32_t* __restrict__ dst, const int32_t* __restrict__ w,
                             int64_t m, int32_t* __restrict__ ew, int32_t* flag) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int32_t a = src[e], b = dst[e], x = w[e];
    if (a < 0 || a >= n || b < 0 || b >= n) {
      atomicOr(flag + 0, 1);
      continue;
    }
    if (x < 0) {
      atomicOr(flag + 1, 1);
      continue;
    }
    if (a == b) continue;  // self-loops are not edges of the graph
    const int64_t pa = row_find(off, adj, a, b), pb = row_find(off, adj, b, a);
    if (pa < 0 || pb < 0) {
      atomicOr(flag + 2, 1);
      continue;
    }
    atomicMax(ew + pa, x);
    atomicMax(ew + pb, x);
  }
}

// One warp per row v: emax[v*L + label(u)] over the row's entries, and the sort keys of the
// edge-weight-ranked segments: (v*L + label(u)) << 32 | (INT32_MAX - w), value = entry index
// (the radix sort is stable, so equal weights keep the id order of the row).
__global__ void k_ew_rows(const int64_t* __restrict__ off, const int32_t* __restrict__ adj,
                          const uint8_t* __restrict__ labels, const int32_t* __restrict__ ew,
                          int32_t n, int32_t L, int32_t* __restrict__ emax,
                          uint64_t* __restrict__ keys, int64_t* __restrict__ vals) {
  const int lane = threadIdx.x & 31;
  for (int64_t v = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; v < n;
       v += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    for (int64_t t = off[v] + lane; t < off[v + 1]; t += 32) {
      const int32_t u = adj[t], x = ew[t], l = labels[u];
      atomicMax(emax + v * L + l, x);
      keys[t] = ((uint64_t)(v * L + l) << 32) | (uint32_t)(INT32_MAX - x);
      vals[t] = t;
    }
  }
}

// lpmax[label(v)*L + l] = max over v of emax[v*L + l] (a plain read first keeps most threads
// off the atomic once the maxima are reached)
__global__ void k_ew_labelpairs(const uint8_t* __restrict__ labels,
                                const int32_t* __restrict__ emax, int32_t n, int32_t L,
                                int32_t* lpmax) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (int64_t)n * L;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t x = emax[i];
    if (x < 0) continue;
    int32_t* cell = lpmax + (int64_t)labels[i / L] * L + (i % L);
    if (x > *(volatile int32_t*)cell) atomicMax(cell, x);
  }
}

__global__ void k_ew_segments(const int64_t* __restrict__ order, int64_t nnz,
                              const int32_t* __restrict__ adj, const int32_t* __restrict__ ew,
                              int2* __restrict__ seg) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nnz;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t t = order[i];
    seg[i] = make_int2(adj[t], ew[t]);
  }
}

}  // namespace

void set_edge_weights(nuri_graph* g, int64_t m, const int32_t* src, const int32_t* dst,
                      const int32_t* w, bool device_input, cudaStream_t s) {
  DevGraph& d = g->d;
  if (!d.lsoff || d.L <= 0)
    NURI_FAIL(NURI_ERR_INVALID,
              "nuri_set_edge_weights: the graph was loaded without labels (or with "
              "NURI_LOAD_NO_ISO): edge-weighted isomorphism needs its label segments");
  const int32_t n = d.n, L = d.L;
  const int64_t nnz = d.nnz;
  DBuf<int32_t> ds, dd, dw;
  const int32_t *ps = src, *pd = dst, *pw = w;
  if (!device_input && m > 0) {
    ds.alloc(m, s);
    dd.alloc(m, s);
    dw.alloc(m, s);
    NURI_CUDA(cudaMemcpyAsync(ds.p, src, sizeof(int32_t) * m, cudaMemcpyHostToDevice, s));
    NURI_CUDA(cudaMemcpyAsync(dd.p, dst, sizeof(int32_t) * m, cudaMemcpyHostToDevice, s));
    NURI_CUDA(cudaMemcpyAsync(dw.p, w, sizeof(int32_t) * m, cudaMemcpyHostToDevice, s));
    ps = ds.p;
    pd = dd.p;
    pw = dw.p;
  }
  DBuf<int32_t> ew, flag;
  ew.alloc(std::max<int64_t>(nnz, 1), s);
  flag.alloc(4, s);
  NURI_CUDA(cudaMemsetAsync(ew.p, 0, sizeof(int32_t) * std::max<int64_t>(nnz, 1), s));
  NURI_CUDA(cudaMemsetAsync(flag.p, 0, 16, s));
  if (m > 0)
    k_ew_scatter<<<blocks_for(m), kThreads, 0, s>>>(g->off.p, g->adj.p, n, ps, pd, pw, m, ew.p,
                                                    flag.p);
  NURI_CUDA(cudaGetLastError());
  int32_t hf[3] = {0, 0, 0};
  NURI_CUDA(cudaMemcpyAsync(hf, flag.p, 12, cudaMemcpyDeviceToHost, s));
  NURI_CUDA(cudaStreamSynchronize(s));
  if (hf[0]) NURI_FAIL(NURI_ERR_INVALID, "nuri_set_edge_weights: vertex id outside [0, n)");
  if (hf[1]) NURI_FAIL(NURI_ERR_INVALID, "nuri_set_edge_weights: negative weight");
  if (hf[2]) NURI_FAIL(NURI_ERR_INVALID, "nuri_set_edge_weights: a pair is not an edge of the graph");
  DBuf<int32_t> emax, lpmax, mx;
  emax.alloc(std::max<int64_t>((int64_t)n * L, 1), s);
  lpmax.alloc((int64_t)L * L, s);
  mx.alloc(1, s);
  NURI_CUDA(cudaMemsetAsync(emax.p, 0xff, sizeof(int32_t) * std::max<int64_t>((int64_t)n * L, 1), s));
  NURI_CUDA(cudaMemsetAsync(lpmax.p, 0xff, sizeof(int32_t) * L * L, s));
  NURI_CUDA(cudaMemsetAsync(mx.p, 0xff, 4, s));
  DBuf<int2> seg;
  seg.alloc(std::max<int64_t>(nnz, 1), s);
  if (nnz > 0) {
    DBuf<uint64_t> k1, k2;
    DBuf<int64_t> v1, v2;
    k1.alloc(nnz, s);
    k2.alloc(nnz, s);
    v1.alloc(nnz, s);
    v2.alloc(nnz, s);
    k_ew_rows<<<std::max(1, std::min(blocks_for((int64_t)n * 32), sm_count() * 32)), kThreads, 0,
                s>>>(g->off.p, g->adj.p, g->labels.p, ew.p, n, L, emax.p, k1.p, v1.p);
    k_ew_labelpairs<<<blocks_for((int64_t)n * L), kThreads, 0, s>>>(g->labels.p, emax.p, n, L,
                                                                    lpmax.p);
    k_max_i32<<<blocks_for(nnz), kThreads, 0, s>>>(ew.p, nnz, mx.p);
    const int end_bit = 32 + bitlen((uint64_t)n * (uint64_t)L);
    size_t tb = 0;
    cub::DeviceRadixSort::SortPairs(nullptr, tb, k1.p, k2.p, v1.p, v2.p, nnz, 0, end_bit, s);
    DBuf<uint8_t> tmp;
    tmp.alloc(tb, s);
    NURI_CUDA(cub::DeviceRadixSort::SortPairs(tmp.p, tb, k1.p, k2.p, v1.p, v2.p, nnz, 0, end_bit,
                                              s));
    k_ew_segments<<<blocks_for(nnz), kThreads, 0, s>>>(v2.p, nnz, g->adj.p, ew.p, seg.p);
    NURI_CUDA(cudaGetLastError());
  }
  int32_t hmax = -1;
  NURI_CUDA(cudaMemcpyAsync(&hmax, mx.p, 4, cudaMemcpyDeviceToHost, s));
  NURI_CUDA(cudaStreamSynchronize(s));
  g->ew = std::move(ew);
  g->emax = std::move(emax);
  g->lpmax = std::move(lpmax);
  g->lseg_e = std::move(seg);
  g->h_ewmax = std::max(hmax, 0);
  d.ew = g->ew.p;
  d.emax = g->emax.p;
  d.lpmax = g->lpmax.p;
  d.lseg_e = g->lseg_e.p;
}

// ---------------------------------------------------------------------------------------------
void build_graph(nuri_graph* g, int32_t n, int64_t m, const int32_t* src, const int32_t* dst,
                 const uint8_t* labels, const int32_t* weights, int32_t index_hops,
                 uint32_t flags, cudaStream_t s) {
  const bool dev_in = flags & NURI_LOAD_DEVICE_INPUT;
  DevGraph& d = g->d;
  d.n = n;
  // 1. inputs on the device
  DBuf<int32_t> dsrc, ddst;
  const int32_t *ps = src, *pd = dst;
  if (!dev_in && m > 0) {
    dsrc.alloc(m, s);
    ddst.alloc(m, s);
    NURI_CUDA(cudaMemcpyAsync(dsrc.p, src, sizeof(int32_t) * m, cudaMemcpyHostToDevice, s));
    NURI_CUDA(cudaMemcpyAsync(ddst.p, dst, sizeof(int32_t) * m, cudaMemcpyHostToDevice, s));
    ps = dsrc.p;
    pd = ddst.p;
  }
  DBuf<int32_t> flag;
  flag.alloc(4, s);
  NURI_CUDA(cudaMemsetAsync(flag.p, 0, 16, s));
  if (m > 0) k_validate<<<blocks_for(m), kThreads, 0, s>>>(ps, pd, m, n, flag.p);
  int32_t bad = 0;
  NURI_CUDA(cudaMemcpyAsync(&bad, flag.p, 4, cudaMemcpyDeviceToHost, s));
  NURI_CUDA(cudaStreamSynchronize(s));
  if (bad) NURI_FAIL(NURI_ERR_INVALID, "nuri_load_graph: vertex id outside [0, n)");

  // 2. sorted, deduplicated directed keys
  DBuf<uint64_t> keys, keys2;
  int64_t two_m = 2 * m;
  int64_t nnz = 0;
  if (two_m > 0) {
    keys.alloc(two_m, s);
    keys2.alloc(two_m, s);
    k_expand_pairs<<<blocks_for(m), kThreads, 0, s>>>(ps, pd, m, n, keys.p);
    int end_bit = 32 + bitlen((uint64_t)n);
    size_t tb = 0;
    cub::DeviceRadixSort::SortKeys(nullptr, tb, keys.p, keys2.p, two_m, 0, end_bit, s);
    DBuf<uint8_t> tmp;
    tmp.alloc(tb, s);
    NURI_CUDA(cub::DeviceRadixSort::SortKeys(tmp.p, tb, keys.p, keys2.p, two_m, 0, end_bit, s));
    DBuf<int64_t> nsel;
    nsel.alloc(1, s);
    size_t tu = 0;
    cub::DeviceSelect::Unique(nullptr, tu, keys2.p, keys.p, nsel.p, two_m, s);
    if (tu > tb) tmp.alloc(tu, s);
    NURI_CUDA(cub::DeviceSelect::Unique(tmp.p, tu, keys2.p, keys.p, nsel.p, two_m, s));
    int64_t nuniq = 0;
    uint64_t last = 0;
    NURI_CUDA(cudaMemcpyAsync(&nuniq, nsel.p, 8, cudaMemcpyDeviceToHost, s));
    NURI_CUDA(cudaStreamSynchronize(s));
    if (nuniq > 0) {
      NURI_CUDA(cudaMemcpyAsync(&last, keys.p + nuniq - 1, 8, cudaMemcpyDeviceToHost, s));
      NURI_CUDA(cudaStreamSynchronize(s));
    }
    nnz = nuniq - ((nuniq > 0 && (last >> 32) == (uint64_t)(uint32_t)n) ? 1 : 0);
  }
  if (nnz >= ((int64_t)1 << 40)) NURI_FAIL(NURI_ERR_LIMIT, "graph too large");
  d.nnz = nnz;
  g->num_edges = nnz / 2;
  g->dropped = m - nnz / 2;

  // CSR
  g->adj.alloc(nnz > 0 ? nnz : 1, s);
  g->deg.alloc(n > 0 ? n : 1, s);
  g->off.alloc((int64_t)n + 1, s);
  NURI_CUDA(cudaMemsetAsync(g->deg.p, 0, sizeof(int32_t) * (n > 0 ? n : 1), s));
  if (nnz > 0) k_split_keys<<<blocks_for(nnz), kThreads, 0, s>>>(keys.p, nnz, g->adj.p, g->deg.p);
  {
    DBuf<int64_t> deg64;
    deg64.alloc((int64_t)n + 1, s);
    NURI_CUDA(cudaMemsetAsync(deg64.p, 0, sizeof(int64_t) * (n + 1), s));
    if (n > 0) k_i32_to_i64<<<blocks_for(n), kThreads, 0, s>>>(g->deg.p, n, deg64.p);
    size_t t = 0;
    cub::DeviceScan::ExclusiveSum(nullptr, t, deg64.p, g->off.p, (int64_t)n + 1, s);
    DBuf<uint8_t> tmp;
    tmp.alloc(t, s);
    NURI_CUDA(cub::DeviceScan::ExclusiveSum(tmp.p, t, deg64.p, g->off.p, (int64_t)n + 1, s));
  }
  d.off = g->off.p;
  d.adj = g->adj.p;
  d.deg = g->deg.p;
  {
    DBuf<int32_t> mx;
    mx.alloc(1, s);
    NURI_CUDA(cudaMemsetAsync(mx.p, 0, 4, s));
    if (n > 0) k_max_i32<<<blocks_for(n), kThreads, 0, s>>>(g->deg.p, n, mx.p);
    NURI_CUDA(cudaMemcpyAsync(&d.max_deg, mx.p, 4, cudaMemcpyDeviceToHost, s));
  }

  // 3. degree orientation (rank space)
  g->vert_of.alloc(n > 0 ? n : 1, s);
  g->rank_of.alloc(n > 0 ? n : 1, s);
  g->ooff.alloc((int64_t)n + 1, s);
  int64_t half = nnz / 2;
  g->oout.alloc(half > 0 ? half : 1, s);
  if (n > 0) {
    DBuf<uint64_t> rk, rk2;
    rk.alloc(n, s);
    rk2.alloc(n, s);
    if (!peel_order(g, rk.p, s))  // very long peels fall back to the (degree, id) order
      k_rank_keys<<<blocks_for(n), kThreads, 0, s>>>(g->deg.p, n, rk.p);
    size_t t = 0;
    cub::DeviceRadixSort::SortKeys(nullptr, t, rk.p, rk2.p, n, 0, 64, s);
    DBuf<uint8_t> tmp;
    tmp.alloc(t, s);
    NURI_CUDA(cub::DeviceRadixSort::SortKeys(tmp.p, t, rk.p, rk2.p, n, 0, 64, s));
    k_rank_split<<<blocks_for(n), kThreads, 0, s>>>(rk2.p, n, g->vert_of.p, g->rank_of.p);
  }
  DBuf<int32_t> odeg;
  odeg.alloc((int64_t)n + 1, s);
  NURI_CUDA(cudaMemsetAsync(odeg.p, 0, sizeof(int32_t) * (n + 1), s));
  if (nnz > 0) {
    k_orient_keys<<<blocks_for(nnz), kThreads, 0, s>>>(keys.p, nnz, g->rank_of.p, n, keys2.p);
    int end_bit = 32 + bitlen((uint64_t)n);
    DBuf<uint64_t> ok2;
    ok2.alloc(nnz, s);
    size_t t = 0;
    cub::DeviceRadixSort::SortKeys(nullptr, t, keys2.p, ok2.p, nnz, 0, end_bit, s);
    DBuf<uint8_t> tmp;
    tmp.alloc(t, s);
    NURI_CUDA(cub::DeviceRadixSort::SortKeys(tmp.p, t, keys2.p, ok2.p, nnz, 0, end_bit, s));
    k_orient_split<<<blocks_for(half), kThreads, 0, s>>>(ok2.p, half, g->oout.p, odeg.p);
  }
  {
    DBuf<int64_t> od64;
    od64.alloc((int64_t)n + 1, s);
    NURI_CUDA(cudaMemsetAsync(od64.p, 0, sizeof(int64_t) * (n + 1), s));
    if (n > 0) k_i32_to_i64<<<blocks_for(n), kThreads, 0, s>>>(odeg.p, n, od64.p);
    size_t t = 0;
    cub::DeviceScan::ExclusiveSum(nullptr, t, od64.p, g->ooff.p, (int64_t)n + 1, s);
    DBuf<uint8_t> tmp;
    tmp.alloc(t, s);
    NURI_CUDA(cub::DeviceScan::ExclusiveSum(tmp.p, t, od64.p, g->ooff.p, (int64_t)n + 1, s));
    DBuf<int32_t> mx;
    mx.alloc(1, s);
    NURI_CUDA(cudaMemsetAsync(mx.p, 0, 4, s));
    if (n > 0) k_max_i32<<<blocks_for(n), kThreads, 0, s>>>(odeg.p, n, mx.p);
    NURI_CUDA(cudaMemcpyAsync(&d.max_out, mx.p, 4, cudaMemcpyDeviceToHost, s));
  }
  d.ooff = g->ooff.p;
  d.oout = g->oout.p;
  d.vert_of = g->vert_of.p;
  d.rank_of = g->rank_of.p;
  // core bitmap of the last ranks (multiple of 64 wide, at most kCoreRanks)
  if (n >= 64 && d.max_out > 64) {
    const int32_t cn = std::min<int32_t>(kCoreRanks, n & ~63);
    g->core_bits.alloc((int64_t)cn * (cn / 64), s);
    NURI_CUDA(cudaMemsetAsync(g->core_bits.p, 0, g->core_bits.bytes(), s));
    k_core_bits<<<std::max(1, std::min(cn / 8, sm_count() * 16)), 256, 0, s>>>(
        g->ooff.p, g->oout.p, n - cn, cn, g->core_bits.p);
    NURI_CUDA(cudaGetLastError());
    d.core_base = n - cn;
    d.core_n = cn;
    d.core_bits = g->core_bits.p;
  }

  // 4. labels, weights, label segments, hop index
  if (weights) {
    g->weights.alloc(n > 0 ? n : 1, s);
    if (n > 0)
      NURI_CUDA(cudaMemcpyAsync(g->weights.p, weights, sizeof(int32_t) * n,
                                dev_in ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
    d.weights = g->weights.p;
    DBuf<int32_t> mn;
    mn.alloc(1, s);
    int32_t init = INT32_MAX;
    NURI_CUDA(cudaMemcpyAsync(mn.p, &init, 4, cudaMemcpyHostToDevice, s));
    if (n > 0) k_min_i32<<<blocks_for(n), kThreads, 0, s>>>(g->weights.p, n, mn.p);
    int32_t wmin = 0;
    NURI_CUDA(cudaMemcpyAsync(&wmin, mn.p, 4, cudaMemcpyDeviceToHost, s));
    NURI_CUDA(cudaStreamSynchronize(s));
    if (n > 0 && wmin < 0) NURI_FAIL(NURI_ERR_INVALID, "nuri_load_graph: negative weight");
  }
  if (labels) {
    g->labels.alloc(n > 0 ? n : 1, s);
    if (n > 0)
      NURI_CUDA(cudaMemcpyAsync(g->labels.p, labels, n,
                                dev_in ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
    d.labels = g->labels.p;
    DBuf<int32_t> mx;
    mx.alloc(1, s);
    NURI_CUDA(cudaMemsetAsync(mx.p, 0, 4, s));
    if (n > 0) k_max_u8<<<blocks_for(n), kThreads, 0, s>>>(g->labels.p, n, mx.p);
    int32_t lmax = 0;
    NURI_CUDA(cudaMemcpyAsync(&lmax, mx.p, 4, cudaMemcpyDeviceToHost, s));
    NURI_CUDA(cudaStreamSynchronize(s));
    d.L = lmax + 1;
  }
  NURI_CUDA(cudaStreamSynchronize(s));
  if (labels && !(flags & NURI_LOAD_NO_ISO) && n > 0) {
    // degree-ranked segments always (patterns and degree-sum isomorphism use them)
    build_label_segments(d, keys.p, g->deg.p, g->lseg_d, &g->lsoff, s);
    d.lsoff = g->lsoff.p;
    d.lseg_d = g->lseg_d.p;
    g->gmax_d.alloc(d.L, s);
    NURI_CUDA(cudaMemsetAsync(g->gmax_d.p, 0xff, sizeof(int32_t) * d.L, s));
    k_gmax<<<blocks_for(n), kThreads, 0, s>>>(g->labels.p, g->deg.p, n, g->gmax_d.p);
    d.gmax_d = g->gmax_d.p;
    if (weights) {
      build_label_segments(d, keys.p, g->weights.p, g->lseg_w, nullptr, s);
      d.lseg_w = g->lseg_w.p;
      g->gmax_w.alloc(d.L, s);
      NURI_CUDA(cudaMemsetAsync(g->gmax_w.p, 0xff, sizeof(int32_t) * d.L, s));
      k_gmax<<<blocks_for(n), kThreads, 0, s>>>(g->labels.p, g->weights.p, n, g->gmax_w.p);
      d.gmax_w = g->gmax_w.p;
    }
    // vertices grouped by label
    {
      DBuf<uint64_t> lk, lk2;
      lk.alloc(n, s);
      lk2.alloc(n, s);
      k_label_keys<<<blocks_for(n), kThreads, 0, s>>>(g->labels.p, n, lk.p);
      size_t t = 0;
      cub::DeviceRadixSort::SortKeys(nullptr, t, lk.p, lk2.p, n, 0, 40, s);
      DBuf<uint8_t> tmp;
      tmp.alloc(t, s);
      NURI_CUDA(cub::DeviceRadixSort::SortKeys(tmp.p, t, lk.p, lk2.p, n, 0, 40, s));
      g->lab_vert.alloc(n, s);
      DBuf<int32_t> cnt;
      cnt.alloc(d.L, s);
      NURI_CUDA(cudaMemsetAsync(cnt.p, 0, sizeof(int32_t) * d.L, s));
      k_label_split<<<blocks_for(n), kThreads, 0, s>>>(lk2.p, n, g->lab_vert.p, cnt.p);
      std::vector<int32_t> hc(d.L);
      NURI_CUDA(cudaMemcpyAsync(hc.data(), cnt.p, sizeof(int32_t) * d.L, cudaMemcpyDeviceToHost, s));
      NURI_CUDA(cudaStreamSynchronize(s));
      g->h_lab_off.assign(d.L + 1, 0);
      for (int l = 0; l < d.L; ++l) g->h_lab_off[l + 1] = g->h_lab_off[l] + hc[l];
      g->lab_off.alloc(d.L + 1, s);
      NURI_CUDA(cudaMemcpyAsync(g->lab_off.p, g->h_lab_off.data(), sizeof(int64_t) * (d.L + 1),
                                cudaMemcpyHostToDevice, s));
      d.lab_off = g->lab_off.p;
      d.lab_vert = g->lab_vert.p;
      g->h_gmax_d.resize(d.L);
      NURI_CUDA(cudaMemcpyAsync(g->h_gmax_d.data(), g->gmax_d.p, sizeof(int32_t) * d.L,
                                cudaMemcpyDeviceToHost, s));
      if (weights) {
        g->h_gmax_w.resize(d.L);
        NURI_CUDA(cudaMemcpyAsync(g->h_gmax_w.data(), g->gmax_w.p, sizeof(int32_t) * d.L,
                                  cudaMemcpyDeviceToHost, s));
      }
      NURI_CUDA(cudaStreamSynchronize(s));
    }
    if (index_hops > 0) {
      d.H = index_hops;
      if (weights) {
        g->idx_w.alloc((int64_t)index_hops * n * d.L, s);
        build_hop_index(d, g->weights.p, index_hops, g->idx_w.p, s);
        d.idx_w = g->idx_w.p;
      }
      g->idx_d.alloc((int64_t)index_hops * n * d.L, s);
      build_hop_index(d, g->deg.p, index_hops, g->idx_d.p, s);
      d.idx_d = g->idx_d.p;
    }
  }
  NURI_CUDA(cudaGetLastError());
  NURI_CUDA(cudaStreamSynchronize(s));
}

}  // namespace nuri

// ---------------------------------------------------------------------------------------------
// Hop/label index without allocation (nuri_hop_index_noalloc).  Some callers cannot allocate
// device memory at the time they need the index: a process whose memory pool is reserved up
// front by another framework, or code running where an allocation could block or fail (a
// latency-bound service thread, a recovery path after an out-of-memory error).  This path
// builds the same index as build_hop_index into the caller's output, on the caller's CSR,
// with the only scratch it needs (the count and list of high-degree vertices, and a flag for
// bad input) held in one fixed array in device memory that the library reserves at load time.
// ---------------------------------------------------------------------------------------------
namespace nuri {
namespace {

// scratch[0]: number of vertices of degree > kHeavy; scratch[1]: bad-input flag;
// scratch[2 ..]: those vertices (at most one per vertex, so NURI_NOALLOC_MAX_VERTICES entries).
// 4 MiB + 8 bytes, held by every GPU that loads the library until the process exits.
static __device__ __align__(256) int32_t g_noalloc_scratch[2 + NURI_NOALLOC_MAX_VERTICES];

// CSR sanity for caller-provided arrays: off[0] = 0, off non-decreasing, off[n] = nnz, every
// neighbour id in [0, n).  Any violation sets flag[0] = 1 (the host then rejects the call).
__global__ void k_check_csr(const int64_t* __restrict__ off, const int32_t* __restrict__ adj,
                            int32_t n, int64_t nnz, int32_t* __restrict__ flag) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t t0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t0 == 0 && (off[0] != 0 || off[n] != nnz)) *flag = 1;
  for (int64_t v = t0; v < n; v += stride)
    if (off[v + 1] < off[v]) *flag = 1;
  for (int64_t i = t0; i < nnz; i += stride) {
    const int32_t x = adj[i];
    if (x < 0 || x >= n) *flag = 1;
  }
}

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
int32_t* g_noalloc_ptr[kMaxDevices] = {};

// Device address of g_noalloc_scratch on the current device (looked up once per device).
int32_t* noalloc_scratch_ptr() {
  int dev = 0;
  NURI_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices)
    NURI_FAIL(NURI_ERR_INVALID, "nuri_hop_index_noalloc: device ordinal %d not supported", dev);
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    int32_t* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress((void**)&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
      NURI_FAIL(NURI_ERR_CUDA, "nuri_hop_index_noalloc: cudaGetSymbolAddress failed (%s)",
                cudaGetErrorName(e));
    g_noalloc_ptr[dev] = p;
  }
  return g_noalloc_ptr[dev];
}

void hop_index_noalloc(int32_t n, const int64_t* off, const int32_t* adj, int64_t nnz,
                       const uint8_t* labels, int32_t L, const int32_t* score, int32_t H,
                       int32_t* out, cudaStream_t s) {
  if (n < 0 || nnz < 0) NURI_FAIL(NURI_ERR_INVALID, "nuri_hop_index_noalloc: negative size");
  if (n > NURI_NOALLOC_MAX_VERTICES)
    NURI_FAIL(NURI_ERR_INVALID,
              "nuri_hop_index_noalloc: %d vertices exceed the limit of %d (the fixed scratch "
              "array holds one entry per vertex)",
              n, NURI_NOALLOC_MAX_VERTICES);
  if (L < 1 || L > 256) NURI_FAIL(NURI_ERR_INVALID, "nuri_hop_index_noalloc: L must be in 1..256");
  if (H < 1 || H > 7) NURI_FAIL(NURI_ERR_INVALID, "nuri_hop_index_noalloc: hops must be in 1..7");
  if (n == 0) return;
  if (!off || !labels || !score || !out || (nnz > 0 && !adj))
    NURI_FAIL(NURI_ERR_INVALID, "nuri_hop_index_noalloc: NULL array");
  int32_t* scratch = noalloc_scratch_ptr();
  int32_t* cnt = scratch;
  int32_t* bad = scratch + 1;
  int32_t* heavy = scratch + 2;
  // the scratch keeps the previous call's contents: the count and the flag start at zero
  NURI_CUDA(cudaMemsetAsync(scratch, 0, 2 * sizeof(int32_t), s));
  k_check_csr<<<sm_count() * 4, kThreads, 0, s>>>(off, adj, n, nnz, bad);
  NURI_CUDA(cudaGetLastError());
  int32_t h[2] = {0, 0};
  NURI_CUDA(cudaMemcpyAsync(h, scratch, 2 * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  NURI_CUDA(cudaStreamSynchronize(s));
  if (h[1]) NURI_FAIL(NURI_ERR_INVALID, "nuri_hop_index_noalloc: malformed CSR (offsets or ids)");
  DevGraph d;
  d.n = n;
  d.nnz = nnz;
  d.L = L;
  d.off = off;
  d.adj = adj;
  d.labels = labels;
  if (L <= 32) {
    k_collect_heavy<<<blocks_for(n), kThreads, 0, s>>>(off, n, heavy, cnt);
    NURI_CUDA(cudaGetLastError());
    NURI_CUDA(cudaMemcpyAsync(h, cnt, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    NURI_CUDA(cudaStreamSynchronize(s));
    const int32_t nheavy = h[0];
    if (L <= 1) hop_rounds_t<1>(d, score, H, out, heavy, nheavy, s);
    else if (L <= 2) hop_rounds_t<2>(d, score, H, out, heavy, nheavy, s);
    else if (L <= 4) hop_rounds_t<4>(d, score, H, out, heavy, nheavy, s);
    else if (L <= 8) hop_rounds_t<8>(d, score, H, out, heavy, nheavy, s);
    else if (L <= 16) hop_rounds_t<16>(d, score, H, out, heavy, nheavy, s);
    else hop_rounds_t<32>(d, score, H, out, heavy, nheavy, s);
  } else {
    for (int h2 = 1; h2 <= H; ++h2) {
      const int32_t* prev = h2 == 1 ? nullptr : out + (int64_t)(h2 - 2) * n * L;
      k_hop_round_generic<<<sm_count() * 8, 256, 0, s>>>(off, adj, labels, score, prev, n, L,
                                                         out + (int64_t)(h2 - 1) * n * L);
    }
  }
  NURI_CUDA(cudaGetLastError());
  NURI_CUDA(cudaStreamSynchronize(s));
}

}  // namespace
}  // namespace nuri

extern "C" nuri_status nuri_hop_index_noalloc(int32_t n, const int64_t* off, const int32_t* adj,
                                              int64_t nnz, const uint8_t* labels, int32_t L,
                                              const int32_t* score, int32_t hops, int32_t* out,
                                              void* stream) {
  try {
    nuri::set_error("%s", "");
    nuri::hop_index_noalloc(n, off, adj, nnz, labels, L, score, hops, out, (cudaStream_t)stream);
    return NURI_OK;
  } catch (const nuri::Err& e) {
    return e.code;
  } catch (...) {
    nuri::set_error("nuri_hop_index_noalloc: unexpected internal error");
    return NURI_ERR_CUDA;
  }
}
