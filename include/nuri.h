/*
 * nuri.h -- C ABI of libnuri, a single-GPU (sm_103a) implementation of prioritized subgraph
 * expansion with pruning for exact top-k subgraph discovery (arXiv 1807.08888, "Nuri").
 *
 * The problem (Section 2, "Top-k Semantics"): given a data graph, a result-set size k and a
 * ranking criterion, return the k most relevant subgraphs without enumerating all of them.
 * Three query kinds are built in, each with the user functions the paper gives for it:
 *   - cliques ranked by size                     (Section 3.2 example, Section 4.1, Listing 1)
 *   - labelled subgraph isomorphism, ranked by the sum of vertex scores
 *                                                (Section 4.3, Listing 3, Fig. 6)
 *   - frequent labelled patterns, ranked by minimum image-based support
 *                                                (Section 2, Section 3.3, Section 4.2, Listing 2)
 *
 * Conventions for every entry point:
 *   - Every function returns a nuri_status; NURI_OK == 0.  On failure a thread-local message
 *     is available from nuri_last_error().  Errors never abort the process and leave the
 *     graph usable.
 *   - Host pointers unless a flag says otherwise.  Inputs are copied; the caller keeps
 *     ownership of everything it passes in.
 *   - `stream` is a cudaStream_t passed as void* (NULL = the legacy default stream).  Every
 *     blocking call enqueues its work on that stream and synchronises it before returning.
 *   - Calls on one nuri_graph are serialised by the caller (one query at a time per graph);
 *     nuri_topk_batch runs many queries in one call.
 *   - Results (nuri_result) are owned by the library and released with nuri_free_result.
 *
 * Ranking and tie-breaking (identical to the CPU oracle): rows are sorted by score descending;
 * equal scores are ordered by the ascending sorted vertex-id list (lexicographic), then, for
 * isomorphism matches, by the ascending sorted edge list, and, for patterns, by the canonical
 * code.  Exactly min(k, number of relevant subgraphs) rows are returned.
 */
#ifndef NURI_H_
#define NURI_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t nuri_status;
#define NURI_OK 0
#define NURI_ERR_INVALID 1   /* bad argument: k < 1, id out of range, bad query, ...      */
#define NURI_ERR_OOM 2       /* device or pinned-host allocation failed                    */
#define NURI_ERR_LIMIT 3     /* a built-in size limit was exceeded (clique size > 256, ...) */
#define NURI_ERR_TIMEOUT 4   /* the query ran past its time budget (nuri_set_time_budget)  */
#define NURI_ERR_CANCELLED 5 /* the request was cancelled                                  */
#define NURI_ERR_CUDA 6      /* a CUDA runtime call failed                                 */
#define NURI_PENDING 7       /* nuri_server_poll: the request has not finished yet         */

/* ranking functions */
#define NURI_RANK_SIZE 0        /* cliques: |V_s|                                           */
#define NURI_RANK_WEIGHT_SUM 1  /* isomorphism, cliques: sum of the int32 vertex weights   */
#define NURI_RANK_DEGREE_SUM 2  /* isomorphism: sum of vertex degrees (the paper's Sec. 6.4) */
#define NURI_RANK_MNI 3         /* patterns: minimum image-based support                   */
#define NURI_RANK_EDGE_WEIGHT_SUM 4 /* isomorphism: sum of the int32 weights of the image's
                                       edges (Section 2's cumulative edge weight)           */

/* nuri_load_graph flags */
#define NURI_LOAD_DEVICE_INPUT 0x1u /* src/dst/labels/weights are device pointers          */
#define NURI_LOAD_NO_ISO 0x2u       /* skip label segments and hop index (cliques only)    */

/* nuri_topk_cliques flags */
#define NURI_CLIQUE_ALL 0x0u        /* every clique is relevant (the paper's relevant()=true) */
#define NURI_CLIQUE_MAXIMAL 0x1u    /* only maximal cliques are relevant                      */
/* flags common to all queries */
#define NURI_KEEP_TIES 0x100u       /* return every row tied with the k-th (|R| may exceed k) */
#define NURI_NO_PRUNE 0x200u        /* disable pruning and prioritization (Nuri-NP ablation)  */
/* nuri_topk_iso flags */
#define NURI_ISO_INDUCED 0x400u     /* induced matches: non-adjacent query vertices map to
                                       non-adjacent data vertices (Section 2's isomorphism
                                       definition read as "edge if and only if edge")       */
/* nuri_topk_patterns flags */
#define NURI_PATTERNS_EDGE_ORIENTED 0x800u /* exhaustive edge-oriented expansion (every connected
                                       M-edge subgraph grown one edge at a time from one-edge
                                       subgraphs, grouped by pattern; Section 2's other
                                       expansion, the Arabesque way): the ablation beside
                                       Algorithm 2, same rows, no pruning                    */

typedef struct nuri_graph nuri_graph;

/* Counters of one query.  "expansions" counts child subgraphs created (Algorithm 1;
 * for patterns, extension candidates examined), including children pruned at once. */
typedef struct nuri_stats {
  int64_t expansions;      /* children created                                   */
  int64_t pruned;          /* children or records dropped by the bound            */
  int64_t dequeued;        /* frontier records / seeds processed                  */
  int64_t spilled;         /* frontier records copied to pinned host memory       */
  int64_t reloaded;        /* spilled records copied back                         */
  int64_t results_stored;  /* candidate results written to the device result set  */
  int64_t rounds;          /* frontier rounds (kernel launches of the expansion)  */
  int64_t adj_bytes;       /* algorithmic bytes of adjacency read by expansions   */
  int64_t threshold;       /* final k-th best score (INT64_MIN if < k results)    */
  int32_t restarts;        /* result-set overflows that forced a re-run          */
  int32_t pad;
  double device_ms;        /* device time from first to last kernel of the query  */
  int64_t launches;        /* kernels of this library launched by the query       */
  int64_t expand_launches; /* launches of the expansion kernel (cliques: also its
                              dense-record launches)                              */
  double expand_ms;        /* summed device time of those launches (CUDA events)  */
  int64_t tail_launches;   /* cliques: launches of the dense-record task kernel    */
  double tail_ms;          /* cliques: summed device time of those launches        */
  int64_t tail_words;      /* cliques: 64-bit adjacency-row words the task kernel
                              combined into candidate masks (colouring, branching) */
  int64_t dense_records[3];/* cliques: records searched on 2-, 4- and 8-word bitmap rows
                              (65..128, 129..256 and 257..512 candidates)           */
  int64_t lex_pruned;      /* cliques: search nodes pruned by the tie bound (their cliques
                              all rank after k known results of the k-th size)      */
} nuri_stats;

/* A result set.  Row i has score[i]; its vertices are verts[vert_off[i] .. vert_off[i+1])
 * (ascending original ids for cliques and isomorphism matches; canonical pattern vertex
 * indices 0..nv-1 for patterns, with labels[] holding each vertex's label); its edges are
 * the pairs edges[2*j], edges[2*j+1] for j in [edge_off[i], edge_off[i+1]) (isomorphism:
 * (min,max) original ids sorted ascending; patterns: canonical index pairs; cliques: none). */
typedef struct nuri_result {
  int32_t count;
  int32_t kind;       /* 0 cliques, 1 isomorphism, 2 patterns */
  int64_t* score;
  int32_t* vert_off;
  int32_t* verts;
  int32_t* edge_off;
  int32_t* edges;
  int32_t* labels;    /* patterns only (NULL otherwise) */
  nuri_stats stats;
} nuri_result;

/* A connected query graph for subgraph isomorphism: nq <= 8 vertices with labels, ne edges
 * given as pairs (src[e], dst[e]) of query vertex indices (host memory). */
typedef struct nuri_query {
  int32_t nq;
  int32_t ne;
  const uint8_t* labels;
  const int32_t* src;
  const int32_t* dst;
} nuri_query;

/* Static facts about a loaded graph. */
typedef struct nuri_graph_info {
  int32_t n;
  int32_t num_labels;    /* 0 when the graph has no labels */
  int64_t num_edges;     /* undirected edges after clean-up */
  int64_t dropped;       /* input pairs dropped (self-loops and duplicates) */
  int32_t max_degree;
  int32_t max_out_degree;/* in the orientation used for cliques: the batch-peeling (core)
                            order, where it equals the degeneracy, or the (degree, id)
                            order when the peel would take over 20000 batches */
  int32_t index_hops;    /* hops of the hop/label index that is resident */
  int32_t pad;
  int64_t device_bytes;  /* device memory held by the graph */
} nuri_graph_info;

/*
 * nuri_load_graph -- build the device-resident graph (Section 5: the engine loads the data
 * graph into memory; Section 4.3: initialize() builds the per-vertex index at load time).
 *   n          number of vertices, ids 0..n-1 (0 <= n < 2^31)
 *   m          number of input pairs; src[e], dst[e] in [0, n).  Undirected: either or both
 *              directions may be given; self-loops and duplicates are dropped.
 *   labels     uint8 per vertex, or NULL (then isomorphism/pattern queries are rejected)
 *   weights    int32 per vertex (>= 0), or NULL (weight-sum ranking then rejected)
 *   index_hops hops H of the hop/label max index to build (0 = none; <= 7).  Queries whose
 *              radius exceeds H fall back to a per-label global maximum for the far vertices.
 *   flags      NURI_LOAD_*
 *   out        receives the graph handle (free with nuri_free_graph)
 * Errors: NURI_ERR_INVALID (bad sizes or ids), NURI_ERR_OOM, NURI_ERR_CUDA.
 */
nuri_status nuri_load_graph(int32_t n, int64_t m, const int32_t* src, const int32_t* dst,
                            const uint8_t* labels, const int32_t* weights, int32_t index_hops,
                            uint32_t flags, void* stream, nuri_graph** out);
void nuri_free_graph(nuri_graph* g);
nuri_status nuri_graph_get_info(const nuri_graph* g, nuri_graph_info* info);

/*
 * nuri_set_edge_weights -- weights of the graph's edges, for isomorphism ranked by cumulative
 * edge weight (NURI_RANK_EDGE_WEIGHT_SUM; Section 2, top-k semantics).
 *   m, src, dst, w  m pairs (src[e], dst[e]) with weight w[e] >= 0, either direction.  An edge
 *          given by several pairs weighs the largest of their weights; an edge given by none
 *          weighs 0; self-loops are ignored.  Host arrays, or device arrays with
 *          NURI_LOAD_DEVICE_INPUT in flags.  Nothing is kept of them after the call.
 *   The call replaces the weights of an earlier call.  The graph must have labels (and its
 *   label segments: not loaded with NURI_LOAD_NO_ISO).  Device memory: 12 bytes per directed
 *   edge entry, plus 4 bytes per (vertex, label) and per label pair.
 * Errors: NURI_ERR_INVALID (a pair that is not an edge of the graph, an id outside [0, n), a
 * negative weight, an unlabelled graph; the graph keeps its previous weights), NURI_ERR_OOM,
 * NURI_ERR_CUDA.
 */
nuri_status nuri_set_edge_weights(nuri_graph* g, int64_t m, const int32_t* src,
                                  const int32_t* dst, const int32_t* w, uint32_t flags,
                                  void* stream);

/*
 * nuri_topk_cliques -- top-k cliques by size (Algorithm 1 with the clique functions of
 * Section 3.2: candidate set P_s of Listing 1 restricted by canonical extension, bound
 * |V_s| + |P_s| (Carraghan-Pardalos), prune a subgraph iff its bound < the k-th best size).
 *   k      >= 1
 *   rank   NURI_RANK_SIZE, or NURI_RANK_WEIGHT_SUM: cliques ranked by the sum of their vertex
 *          weights (graph loaded with weights), bound w(V_s) + w(P_s), ties by sorted ids
 *          (Section 2 leaves the ranking criterion to the user; frontier_cap is not used)
 *   flags  NURI_CLIQUE_ALL (default: every clique, singletons included, is a result) or
 *          NURI_CLIQUE_MAXIMAL; optionally NURI_KEEP_TIES, NURI_NO_PRUNE
 *   frontier_cap  maximum number of frontier records kept on the device before the lowest
 *          buckets are spilled to pinned host memory (0 = library default)
 * Errors: NURI_ERR_INVALID, NURI_ERR_LIMIT (a clique larger than 256), NURI_ERR_OOM, CUDA.
 */
nuri_status nuri_topk_cliques(nuri_graph* g, int32_t k, int32_t rank, uint32_t flags,
                              int64_t frontier_cap, void* stream, nuri_result** out);

/*
 * nuri_topk_iso -- top-k subgraphs isomorphic to a query (Section 2 definition, non-induced
 * image subgraphs; Section 4.3 functions: score = sum of vertex scores, upper bound =
 * score + sum over unmatched query vertices of index(root image, label, hop)).
 *   rank   NURI_RANK_WEIGHT_SUM or NURI_RANK_DEGREE_SUM, or NURI_RANK_EDGE_WEIGHT_SUM (score =
 *          sum of the weights of the image's edges, nuri_set_edge_weights; upper bound =
 *          score + for each unmatched query edge the largest weight an edge between its
 *          endpoints' images could have: from a matched image, its heaviest edge to the
 *          label; otherwise the heaviest edge between the two labels)
 *   flags  NURI_KEEP_TIES, NURI_ISO_INDUCED (induced matches only)
 * Errors: NURI_ERR_INVALID (nq outside 1..8, disconnected query, no labels/weights/edge
 * weights for the rank asked).
 */
nuri_status nuri_topk_iso(nuri_graph* g, const nuri_query* q, int32_t k, int32_t rank,
                          uint32_t flags, void* stream, nuri_result** out);

/*
 * nuri_topk_iso_batch -- nqueries isomorphism queries in one call; the seeds and frontiers of
 * all queries are expanded together by the same kernels.  outs[i] receives query i's result.
 * At most 4095 queries a call (NURI_ERR_LIMIT above).
 */
nuri_status nuri_topk_iso_batch(nuri_graph* g, int32_t nqueries, const nuri_query* qs,
                                const int32_t* ks, int32_t rank, uint32_t flags, void* stream,
                                nuri_result** outs);

/*
 * nuri_topk_patterns -- top-k connected vertex-labelled patterns with exactly M edges by
 * minimum image-based support (Algorithm 2, Section 4.2 functions: priority (m, f),
 * dominated = f < f(k-th)).  1 <= M <= 5.
 *   flags  NURI_KEEP_TIES; NURI_PATTERNS_EDGE_ORIENTED computes the same rows by exhaustive
 *          edge-oriented expansion (stats.expansions = subgraphs grown, stats.results_stored =
 *          embeddings, stats.dequeued = distinct patterns); NURI_ERR_LIMIT when more than 4096
 *          edges touch one subgraph or the embeddings pass 2^28.
 */
nuri_status nuri_topk_patterns(nuri_graph* g, int32_t M, int32_t k, int32_t rank,
                               uint32_t flags, void* stream, nuri_result** out);

/*
 * nuri_hop_index -- copy the resident hop/label index to the caller: out[((h-1)*n+v)*L+l]
 * = max weight (or degree if degree_rank) over vertices of label l reachable from v by a walk
 * of 1..h edges, -1 when there is none (Section 4.3, Listing 3; cumulative-hop reading).
 * `out` is a device pointer when `device_out` is non-zero, else host.  hops <= index_hops.
 */
nuri_status nuri_hop_index(nuri_graph* g, int32_t hops, int32_t degree_rank, int32_t* out,
                           int32_t device_out, void* stream);

/*
 * nuri_hop_index_noalloc -- the hop/label index of nuri_hop_index, built on a graph the caller
 * already holds on the device, with no memory allocated by this call.  The paper has no
 * counterpart: this entry point exists for callers that cannot allocate device memory when
 * they need the index (a process whose GPU memory another framework has reserved up front,
 * a service thread that must not block or fail inside an allocator, a recovery path after an
 * out-of-memory error).
 *
 *   n       vertices, 0 <= n <= NURI_NOALLOC_MAX_VERTICES (larger n: NURI_ERR_INVALID)
 *   off     device int64[n + 1] CSR row offsets, off[0] = 0, off[n] = nnz
 *   adj     device int32[nnz] neighbour ids in [0, n); each undirected edge in both rows, no
 *           self-loops, no duplicates (the adjacency nuri_load_graph builds)
 *   labels  device uint8[n], values < L;  score  device int32[n], >= 0 (weights or degrees)
 *   L       labels, 1..256;  hops  1..7
 *   out     device int32[hops * n * L]: out[((h-1)*n + v)*L + l] as in nuri_hop_index
 *   stream  CUDA stream (NULL: the legacy default stream); the call returns after the
 *           stream has finished the work
 * Scratch: one fixed device array of NURI_NOALLOC_MAX_VERTICES + 2 int32 (4 MiB) that the
 * library holds on every GPU where it is loaded, until the process exits.  Every call shares
 * it and it keeps the previous call's contents (the call clears what must start at zero), so
 * calls that overlap on the GPU (several streams, threads or processes sharing the context)
 * race: serialise them.  The first call on each device looks up that array's device address
 * (which may make the driver load the library's device code): make the first call on a
 * device before any stream capture and outside any section that must not allocate.
 * Errors: NURI_ERR_INVALID (sizes, NULL arrays, or a CSR that fails the offset/id check,
 * which runs on the device before the index), NURI_ERR_CUDA.  Nothing is written to `out`
 * when the call is rejected.
 */
#define NURI_NOALLOC_MAX_VERTICES (1 << 20)
nuri_status nuri_hop_index_noalloc(int32_t n, const int64_t* off, const int32_t* adj,
                                   int64_t nnz, const uint8_t* labels, int32_t L,
                                   const int32_t* score, int32_t hops, int32_t* out,
                                   void* stream);

/*
 * Seed partition: one query split over several GPUs (or processes), each running the same
 * query on a copy of the graph with a part of the seeds.  Algorithm 1's seeds are independent
 * units (Section 3.2: every subgraph grows from one unit subgraph), so the parts share
 * nothing but the threshold: each part only needs to know that the k-th best score is at
 * least some value to prune with it.
 *   index, count  this part and the number of parts (count = 1: no partition).  A seed
 *                 belongs to part nuri_seed_part(v, count), v its original vertex id: for
 *                 cliques the vertex every clique below the seed starts from (its first
 *                 vertex in the library's canonical order), for isomorphism the data vertex
 *                 the query's root is mapped to.
 *   exchange      called on the host between rounds (cliques: every frontier round;
 *                 isomorphism: between seed chunks) with the query index in its batch and
 *                 the part's current threshold (INT64_MIN while it has fewer than k rows);
 *                 returns the largest threshold any part has published so far (which the
 *                 part then prunes with).  It must not wait for the other parts: parts run
 *                 different numbers of rounds.  NULL: no exchange.
 * A partitioned query returns the part's own top k: every row of the global top k whose
 * seed lies in the part, with the same ranking; merging the parts' rows by the ranking and
 * keeping k gives the global answer.  The query's other counters are the part's own.
 */
typedef int64_t (*nuri_tau_exchange_fn)(void* ctx, int32_t query, int64_t local_tau);
typedef struct nuri_partition {
  int32_t index;
  int32_t count;
  nuri_tau_exchange_fn exchange;
  void* ctx;
} nuri_partition;

/* Set (or, with p = NULL or p->count == 1, clear) the seed partition of every later clique
 * and isomorphism query on g.  Errors: NURI_ERR_INVALID (count < 1, index outside
 * 0..count-1). */
nuri_status nuri_set_partition(nuri_graph* g, const nuri_partition* p);

/* The part a seed vertex id belongs to among `count` parts: a fixed integer mix of v (the
 * 32-bit finaliser of MurmurHash3) modulo count.  Host function; needs no GPU. */
int32_t nuri_seed_part(int32_t v, int32_t count);

/*
 * nuri_tune_cliques -- autotune the dense-record search of top-k clique queries on this graph
 * (the batched form's work granularity; no counterpart in the paper, whose search is
 * sequential).  Runs the query (g, k, flags) once per candidate task granularity (48, 96,
 * 128, 192: search nodes with more candidates than this become tasks of the global queue),
 * times each with the device timer and keeps the fastest for every later nuri_topk_cliques
 * call on g.  Results never depend on the setting.  *chosen (may be NULL) receives it and
 * *best_ms (may be NULL) its device time.  The environment variable NURI_TASK_SPLIT, when
 * set, still overrides the tuned value.  Errors: those of nuri_topk_cliques (the previous
 * setting is kept).
 */
nuri_status nuri_tune_cliques(nuri_graph* g, int32_t k, uint32_t flags, void* stream,
                              int32_t* chosen, double* best_ms);

/*
 * nuri_set_time_budget -- limit the device time of every later query on any graph: a query
 * whose kernels run past `ms` milliseconds stops and returns NURI_ERR_TIMEOUT (the graph
 * stays usable).  The check reads the GPU's global timer inside the search loops; no kernel
 * waits on anything.  0 (the default) means no limit.  Process-wide setting.
 */
nuri_status nuri_set_time_budget(double ms);

void nuri_free_result(nuri_result* r);

/* ---- serving: continuous batching over one resident graph ------------------------------ */

#define NURI_REQ_CLIQUES 0
#define NURI_REQ_ISO 1
#define NURI_REQ_PATTERNS 2

/* One request: kind NURI_REQ_CLIQUES (rank NURI_RANK_SIZE, flags as nuri_topk_cliques),
 * NURI_REQ_ISO (query, rank WEIGHT_SUM or DEGREE_SUM, flags as nuri_topk_iso) or
 * NURI_REQ_PATTERNS (pattern_edges = M in 1..5, rank NURI_RANK_MNI; nuri_topk_batch only).
 * The query arrays are copied at submission. */
typedef struct nuri_request {
  int32_t kind;
  int32_t k;
  int32_t rank;
  uint32_t flags;
  nuri_query query;
  int32_t pattern_edges;
  int32_t pad;
} nuri_request;

/*
 * nuri_topk_batch -- many top-k requests of any kind on one graph in one call (Algorithm 1 /
 * Algorithm 2 run per query, Section 3; the batched form of the engine).  outs[i] receives
 * request i's result, exactly what the request alone returns (rows; the counters in `stats`
 * are those of the shared work that produced it).  How requests share work:
 *   - cliques with equal flags: the ranking (size desc, sorted ids asc) does not depend on
 *     k, so every request's rows are a prefix of the top-K list, K = the largest k of the
 *     group; one search with K answers them all (with NURI_KEEP_TIES: one search keeping
 *     ties, each request keeping the rows that tie with its own k-th);
 *   - patterns with equal M and flags: the same, one Algorithm 2 run per M;
 *   - isomorphism requests with equal rank and flags: one batched launch, as
 *     nuri_topk_iso_batch (every query keeps its own frontier and threshold).
 * Errors: NURI_ERR_INVALID (a bad request: unknown kind, k < 1, bad query, M outside 1..5),
 * or the first error of a query run; on any error every outs[i] is NULL.
 */
nuri_status nuri_topk_batch(nuri_graph* g, int32_t nreq, const nuri_request* reqs,
                            void* stream, nuri_result** outs);

/* slots: concurrent requests (one CUDA stream and one host worker each, default 4);
 * max_batch: isomorphism requests merged into one launch (default 64);
 * mem_budget_bytes: device memory admitted requests may hold together, plus the clique
 * kernels' local memory that the driver reserves once per context (0: 80 % of the device
 * memory free when the server is created). */
typedef struct nuri_server_cfg {
  int32_t slots;
  int32_t max_batch;
  int64_t mem_budget_bytes;
} nuri_server_cfg;

/* Host-clock times of a finished request: waiting for admission, running, and both; the
 * start and end of its service on the host's monotonic clock (milliseconds, any origin;
 * comparable between requests of one process); and the device bytes it was admitted with. */
typedef struct nuri_request_times {
  double queue_ms;
  double service_ms;
  double total_ms;
  double start_ms;
  double done_ms;
  int64_t mem_bytes;
} nuri_request_times;

typedef struct nuri_server nuri_server;

/*
 * nuri_server_create -- start a request server on a loaded graph (the graph must outlive it).
 * Requests are admitted oldest first as soon as a slot is free and their device-memory
 * estimate (nuri_request_bytes) fits the budget; requests waiting together run as one
 * nuri_topk_batch call: isomorphism requests as one batched launch, clique requests with the
 * same flags as one shared search.  Results are identical to the same query run alone.
 */
nuri_status nuri_server_create(nuri_graph* g, const nuri_server_cfg* cfg, nuri_server** out);
/* Queue a request (thread-safe); *ticket identifies it. */
nuri_status nuri_server_submit(nuri_server* s, const nuri_request* r, uint64_t* ticket);
/* Non-blocking: NURI_PENDING while running; otherwise the request's status, its result in
 * *out (caller frees with nuri_free_result) and its times (times may be NULL).  A ticket is
 * reported once. */
nuri_status nuri_server_poll(nuri_server* s, uint64_t ticket, nuri_result** out,
                             nuri_request_times* times);
/* Blocking variant of nuri_server_poll. */
nuri_status nuri_server_wait(nuri_server* s, uint64_t ticket, nuri_result** out,
                             nuri_request_times* times);
/* Number of batched isomorphism launches and of requests they carried. */
nuri_status nuri_server_stats(nuri_server* s, int64_t* batches, int64_t* batched);
/* Number of shared clique searches and of clique requests they answered. */
nuri_status nuri_server_clique_stats(nuri_server* s, int64_t* searches, int64_t* requests);
/* The server's device-memory budget and the part of it held for the whole run (the clique
 * kernels' local memory, reserved once per context); either pointer may be NULL. */
nuri_status nuri_server_budget(nuri_server* s, int64_t* budget_bytes, int64_t* fixed_bytes);

/*
 * nuri_request_bytes -- the device memory a request may hold while it runs: an upper bound of
 * every buffer its query allocates on graph g (for cliques: seeds, staging, the device
 * frontier at its default capacity, round arrays, split-tier scratch, dense-record stores
 * and task queues at their maximum, the initial result set and the final merge; for
 * isomorphism: seeds, result region, selection and merge).  This is the figure the server
 * admits requests by.  A clique result set that outgrows its initial size (compaction keeps
 * it to the rows at or above the threshold first) adds to it.
 * Errors: NURI_ERR_INVALID (NULL arguments, k < 1, unknown kind).
 */
nuri_status nuri_request_bytes(const nuri_graph* g, const nuri_request* r, int64_t* bytes);
/* Finish every queued request, stop the workers, free unclaimed results. */
void nuri_server_destroy(nuri_server* s);

/* Message of the last failure on the calling thread ("" if none). */
const char* nuri_last_error(void);

/* Library version string. */
const char* nuri_version(void);

#ifdef __cplusplus
}
#endif

#endif /* NURI_H_ */
