// Internal declarations shared by the translation units of libnuri.
#pragma once

#include <cuda_runtime.h>
#include <atomic>
#include <cstdint>
#include <string>
#include <vector>

#include "nuri.h"

namespace nuri {

// ------------------------------------------------------------------------------------------
// errors
// ------------------------------------------------------------------------------------------
void set_error(const char* fmt, ...);
const char* last_error();

struct Err {
  nuri_status code;
};

// Source line of the last CUDA call made through NURI_CUDA (any thread): read only by the
// query watchdog's report.
extern std::atomic<int> g_cuda_site;

// Throws Err on a CUDA failure; every C entry point catches and converts to a status.
#define NURI_CUDA(call)                                                                    \
  do {                                                                                    \
    ::nuri::g_cuda_site.store(__LINE__, std::memory_order_relaxed);                       \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess) {                                                              \
      ::nuri::set_error("CUDA error %s at %s:%d: %s", cudaGetErrorName(e_), __FILE__,     \
                        __LINE__, cudaGetErrorString(e_));                                \
      throw ::nuri::Err{e_ == cudaErrorMemoryAllocation ? NURI_ERR_OOM : NURI_ERR_CUDA};  \
    }                                                                                     \
  } while (0)

#define NURI_FAIL(code, ...)          \
  do {                                \
    ::nuri::set_error(__VA_ARGS__);   \
    throw ::nuri::Err{code};          \
  } while (0)

// ------------------------------------------------------------------------------------------
// stream-ordered device buffers
// ------------------------------------------------------------------------------------------
// The library's memory pool on the current device (capi.cu): freed blocks stay cached in it,
// up to a bound, so that the buffers of one query are reused by the next without going back
// to the driver.
cudaMemPool_t device_pool();

template <class T>
struct DBuf {
  T* p = nullptr;
  size_t n = 0;
  cudaStream_t s = nullptr;
  DBuf() = default;
  DBuf(const DBuf&) = delete;
  DBuf& operator=(const DBuf&) = delete;
  DBuf(DBuf&& o) noexcept { swap(o); }
  DBuf& operator=(DBuf&& o) noexcept {
    reset();
    swap(o);
    return *this;
  }
  ~DBuf() { reset(); }
  void swap(DBuf& o) {
    std::swap(p, o.p);
    std::swap(n, o.n);
    std::swap(s, o.s);
  }
  void alloc(size_t count, cudaStream_t st) {
    reset();
    s = st;
    n = count;
    if (count) NURI_CUDA(cudaMallocFromPoolAsync((void**)&p, sizeof(T) * count, device_pool(), st));
  }
  void reset() {
    if (p) cudaFreeAsync(p, s);
    p = nullptr;
    n = 0;
  }
  size_t bytes() const { return sizeof(T) * n; }
};

// ------------------------------------------------------------------------------------------
// the device-resident graph
// ------------------------------------------------------------------------------------------
// Layouts (all int32 vertex ids, int64 row offsets):
//   adj      : undirected CSR, each row sorted by id                  off[n+1], adj[2|E|]
//   orientation for cliques: rank(v) = position of v in the degeneracy (batch-peeling) order;
//     oout   : out-rows in rank space, row r = ranks of neighbours with larger rank, sorted
//     vert_of: rank -> original id
//   label segments for isomorphism / patterns: the row of v is grouped by neighbour label;
//     segment (v, l) = lseg[lsoff[v*L + l] .. lsoff[v*L + l + 1]) holds {id, score} pairs
//     sorted by score descending, then id ascending (weight-ranked candidate lists)
//   hop index: idx[((h-1) * n + v) * L + l], h = 1..H (cumulative walk reachability)
struct DevGraph {
  int32_t n = 0;
  int64_t nnz = 0;        // directed entries = 2|E|
  int32_t L = 0;          // number of labels (0 = unlabelled)
  int32_t max_deg = 0, max_out = 0;
  const int64_t* off = nullptr;
  const int32_t* adj = nullptr;
  const int32_t* deg = nullptr;
  const int64_t* ooff = nullptr;
  const int32_t* oout = nullptr;
  const int32_t* vert_of = nullptr;
  const int32_t* rank_of = nullptr;
  // core bitmap: adjacency of the last core_n ranks (the densest core of the degeneracy
  // order), row r - core_base = core_n/64 words; bit (a, b) set iff ranks a, b are adjacent
  int32_t core_base = 0, core_n = 0;
  const unsigned long long* core_bits = nullptr;
  const uint8_t* labels = nullptr;
  const int32_t* weights = nullptr;
  const int64_t* lsoff = nullptr;   // [n*L + 1]
  const int2* lseg_w = nullptr;     // weight-ranked segments {id, weight}
  const int2* lseg_d = nullptr;     // degree-ranked segments {id, degree}
  const int32_t* idx_w = nullptr;   // hop index over weights
  const int32_t* idx_d = nullptr;   // hop index over degrees
  const int32_t* gmax_w = nullptr;  // [L] global per-label max weight
  const int32_t* gmax_d = nullptr;  // [L] global per-label max degree
  const int64_t* lab_off = nullptr; // [L+1] vertices grouped by label
  const int32_t* lab_vert = nullptr;// [n]   (ascending id inside a label)
  int32_t H = 0;
  // edge weights (nuri_set_edge_weights): ew[t] = weight of CSR entry t (both directions of an
  // edge hold the same value); emax[v*L + l] = largest weight of an edge from v to a neighbour
  // of label l (-1: none); lpmax[a*L + b] = largest weight of an edge between labels a and b
  // (-1: none); lseg_e: the label segments (same lsoff) as {id, w(v, id)}, weight descending
  const int32_t* ew = nullptr;
  const int32_t* emax = nullptr;
  const int32_t* lpmax = nullptr;
  const int2* lseg_e = nullptr;
};

}  // namespace nuri

struct nuri_graph {
  nuri::DevGraph d;
  nuri_partition part{0, 1, nullptr, nullptr};  // seed partition of later queries
  int64_t num_edges = 0, dropped = 0;
  int32_t degeneracy = -1;  // from the peeling order (-1: degree order used)
  int32_t clique_split_bits = 0;  // dense-search task granularity chosen by nuri_tune_cliques
  cudaStream_t stream = nullptr;
  nuri::DBuf<int64_t> off, ooff, lsoff, lab_off;
  nuri::DBuf<int32_t> adj, deg, oout, vert_of, rank_of, weights, idx_w, idx_d, gmax_w, gmax_d;
  nuri::DBuf<unsigned long long> core_bits;
  nuri::DBuf<uint8_t> labels;
  nuri::DBuf<int32_t> lab_vert;
  std::vector<int32_t> h_gmax_w, h_gmax_d;  // host copies of the per-label maxima
  std::vector<int64_t> h_lab_off;           // host copy of lab_off
  nuri::DBuf<int2> lseg_w, lseg_d;
  nuri::DBuf<int32_t> ew, emax, lpmax;  // edge weights and their maxima
  nuri::DBuf<int2> lseg_e;
  int32_t h_ewmax = -1;                 // largest edge weight (-1: no edge weights set)
  int64_t device_bytes() const {
    return off.bytes() + ooff.bytes() + lsoff.bytes() + adj.bytes() + deg.bytes() +
           oout.bytes() + vert_of.bytes() + rank_of.bytes() + weights.bytes() + idx_w.bytes() +
           idx_d.bytes() + gmax_w.bytes() + gmax_d.bytes() + labels.bytes() + lseg_w.bytes() +
           lseg_d.bytes() + lab_off.bytes() + lab_vert.bytes() + core_bits.bytes() +
           ew.bytes() + emax.bytes() + lpmax.bytes() + lseg_e.bytes();
  }
};

namespace nuri {

// The part of a seed vertex among `count` parts (MurmurHash3's 32-bit finaliser, mod count).
__host__ __device__ __forceinline__ int32_t seed_part(int32_t v, int32_t count) {
  uint32_t x = (uint32_t)v;
  x ^= x >> 16;
  x *= 0x85ebca6bu;
  x ^= x >> 13;
  x *= 0xc2b2ae35u;
  x ^= x >> 16;
  return count <= 1 ? 0 : (int32_t)(x % (uint32_t)count);
}

// graph_build.cu
void build_graph(nuri_graph* g, int32_t n, int64_t m, const int32_t* src, const int32_t* dst,
                 const uint8_t* labels, const int32_t* weights, int32_t index_hops,
                 uint32_t flags, cudaStream_t s);

// edge weights of a loaded graph (graph_build.cu): m pairs (src, dst) with weight w >= 0, on
// the host or (device_input) on the device; every pair must be an edge of the graph
void set_edge_weights(nuri_graph* g, int64_t m, const int32_t* src, const int32_t* dst,
                      const int32_t* w, bool device_input, cudaStream_t s);

// result packing (capi.cu)
nuri_result* new_result(int kind, int32_t count, int64_t nverts, int64_t nedges, bool labels);

// cliques.cu
void topk_cliques(nuri_graph* g, int32_t k, uint32_t flags, int64_t frontier_cap,
                  cudaStream_t s, nuri_result** out);

// wcliques.cu: cliques ranked by cumulative vertex weight, and its device memory bound
void topk_wcliques(nuri_graph* g, int32_t k, uint32_t flags, cudaStream_t s, nuri_result** out);
int64_t wclique_query_bytes(const nuri_graph* g, int32_t k);

// device bytes one clique query may allocate, and the local memory of the clique kernels
int64_t clique_query_bytes(const nuri_graph* g, int32_t k, uint32_t flags, int64_t frontier_cap);
int64_t clique_local_reserve_bytes();

// server.cu: device bytes a request may hold while it runs
int64_t request_bytes(const nuri_graph* g, const nuri_request& r);

// iso.cu
int64_t iso_query_bytes(const nuri_graph* g, int32_t k);
void topk_iso_batch(nuri_graph* g, int32_t nq, const nuri_query* qs, const int32_t* ks,
                    int32_t rank, uint32_t flags, cudaStream_t s, nuri_result** outs);

// patterns.cu
void topk_patterns(nuri_graph* g, int32_t M, int32_t k, uint32_t flags, cudaStream_t s,
                   nuri_result** out);

// timing helper: device events on the query stream
struct DevTimer {
  cudaEvent_t a = nullptr, b = nullptr;
  cudaStream_t s;
  explicit DevTimer(cudaStream_t st) : s(st) {
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    cudaEventRecord(a, s);
  }
  double stop() {
    cudaEventRecord(b, s);
    cudaEventSynchronize(b);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    return ms;
  }
  ~DevTimer() {
    cudaEventDestroy(a);
    cudaEventDestroy(b);
  }
};

// process-wide query time budget in nanoseconds (0 = none), set by nuri_set_time_budget
uint64_t time_budget_ns();

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

// writes *deadline = now + budget (or ~0 when budget == 0); launched first by every query
__global__ void k_set_deadline(uint64_t* deadline, uint64_t budget_ns);

inline int sm_count() {
  static int c = 0;
  if (!c) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&c, cudaDevAttrMultiProcessorCount, dev);
    if (c <= 0) c = 148;
  }
  return c;
}

}  // namespace nuri
