// Continuous-batching request server over one resident graph.
//
// Requests (top-k cliques or top-k isomorphism) are submitted from any thread and return a
// ticket.  `slots` worker threads each own a CUDA stream; a worker takes the oldest pending
// request whose memory estimate fits the free part of the device-memory budget, and every
// other pending request of the same kind and settings (up to max_batch): isomorphism queries
// with the same score mode then run as one batched launch, clique requests as one shared
// search whose largest k answers all of them (nuri_topk_batch).  Requests that arrive
// while others run are admitted as soon as a slot and memory free up, so the work of many
// requests overlaps on the device (different streams).  Each request's result is the same as
// when it runs alone: queries share only the read-only graph.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <set>
#include <thread>
#include <vector>

#include "nuri_internal.cuh"

struct nuri_server {
  nuri_graph* g = nullptr;
  nuri_server_cfg cfg{};
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  struct Req {
    uint64_t ticket;
    nuri_request r;
    std::vector<uint8_t> qlab;
    std::vector<int32_t> qsrc, qdst;
    int64_t mem;
    double t_submit;
  };
  struct Done {
    nuri_status status;
    nuri_result* res;
    std::string err;
    double t_submit, t_start, t_done;
    int64_t mem;
  };
  std::deque<Req> pending;
  std::map<uint64_t, Done> done;
  std::set<uint64_t> live;  // submitted tickets not yet reported
  std::vector<std::thread> workers;
  std::vector<cudaStream_t> streams;
  int64_t mem_in_use = 0;
  int64_t fixed_bytes = 0;  // local memory of the clique kernels, reserved once per context
  uint64_t next_ticket = 1;
  bool stopping = false;
  std::atomic<int64_t> n_batches{0}, n_batched{0};              // isomorphism launches
  std::atomic<int64_t> n_clique_batches{0}, n_clique_batched{0};  // shared clique searches
};

namespace nuri {
namespace {

double now_ms() {
  return std::chrono::duration<double, std::milli>(
             std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

}  // namespace
}  // namespace nuri

// device memory a request may hold while it runs: the upper bound of every buffer its query
// allocates (nuri_request_bytes)
int64_t nuri::request_bytes(const nuri_graph* g, const nuri_request& r) {
  if (r.kind == NURI_REQ_CLIQUES)
    return r.rank == NURI_RANK_WEIGHT_SUM ? wclique_query_bytes(g, r.k)
                                          : clique_query_bytes(g, r.k, r.flags, 0);
  return iso_query_bytes(g, r.k);
}

namespace nuri {
namespace {

void worker_main(nuri_server* S, int slot) {
  cudaStream_t st = S->streams[slot];
  int dev = 0;
  cudaGetDevice(&dev);
  while (true) {
    std::vector<nuri_server::Req> batch;
    int64_t mem = 0;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      while (true) {
        if (S->stopping && S->pending.empty()) return;
        // the oldest request that fits the free memory (first-come first-served otherwise);
        // a request larger than the whole budget runs alone
        auto it = S->pending.begin();
        for (; it != S->pending.end(); ++it)
          if (S->fixed_bytes + S->mem_in_use + it->mem <= S->cfg.mem_budget_bytes ||
              S->mem_in_use == 0)
            break;
        if (it != S->pending.end()) {
          batch.push_back(std::move(*it));
          S->pending.erase(it);
          mem = batch[0].mem;
          if (batch[0].r.kind == NURI_REQ_CLIQUES) {
            // clique requests with the same flags share one search (the largest k answers
            // every smaller one): the group holds the memory of its largest request
            for (auto jt = S->pending.begin();
                 jt != S->pending.end() && (int)batch.size() < S->cfg.max_batch;) {
              if (jt->r.kind == NURI_REQ_CLIQUES && jt->r.flags == batch[0].r.flags &&
                  jt->r.rank == batch[0].r.rank &&
                  S->fixed_bytes + S->mem_in_use + std::max(mem, jt->mem) <=
                      S->cfg.mem_budget_bytes) {
                mem = std::max(mem, jt->mem);
                batch.push_back(std::move(*jt));
                jt = S->pending.erase(jt);
              } else {
                ++jt;
              }
            }
          }
          if (batch[0].r.kind == NURI_REQ_ISO) {
            for (auto jt = S->pending.begin();
                 jt != S->pending.end() && (int)batch.size() < S->cfg.max_batch;) {
              if (jt->r.kind == NURI_REQ_ISO && jt->r.rank == batch[0].r.rank &&
                  jt->r.flags == batch[0].r.flags &&
                  S->fixed_bytes + S->mem_in_use + mem + jt->mem <= S->cfg.mem_budget_bytes) {
                mem += jt->mem;
                batch.push_back(std::move(*jt));
                jt = S->pending.erase(jt);
              } else {
                ++jt;
              }
            }
          }
          S->mem_in_use += mem;
          break;
        }
        S->cv_work.wait(lk);
      }
    }
    double t_start = now_ms();
    std::vector<nuri_status> status(batch.size(), NURI_OK);
    std::vector<nuri_result*> res(batch.size(), nullptr);
    std::vector<std::string> err(batch.size());
    cudaSetDevice(dev);
    {
      // one nuri_topk_batch call: an isomorphism group is one batched launch, a clique group
      // one shared search
      std::vector<nuri_request> rq(batch.size());
      for (size_t i = 0; i < batch.size(); ++i) {
        rq[i] = batch[i].r;
        if (rq[i].kind == NURI_REQ_ISO) {
          rq[i].query.labels = batch[i].qlab.data();
          rq[i].query.src = batch[i].qsrc.data();
          rq[i].query.dst = batch[i].qdst.data();
        }
      }
      nuri_status rc = nuri_topk_batch(S->g, (int32_t)rq.size(), rq.data(), st, res.data());
      if (rc) {
        std::string e = nuri_last_error();
        for (size_t i = 0; i < batch.size(); ++i) {
          status[i] = rc;
          err[i] = e;
        }
      }
      if (batch[0].r.kind == NURI_REQ_ISO) {
        S->n_batches += 1;
        S->n_batched += (int64_t)batch.size();
      } else {
        S->n_clique_batches += 1;
        S->n_clique_batched += (int64_t)batch.size();
      }
    }
    double t_done = now_ms();
    {
      std::lock_guard<std::mutex> lk(S->mu);
      S->mem_in_use -= mem;
      for (size_t i = 0; i < batch.size(); ++i)
        S->done[batch[i].ticket] = {status[i], res[i],       err[i],       batch[i].t_submit,
                                    t_start,   t_done,       batch[i].mem};
    }
    S->cv_done.notify_all();
    S->cv_work.notify_all();
  }
}

}  // namespace
}  // namespace nuri

using namespace nuri;

extern "C" {

nuri_status nuri_server_create(nuri_graph* g, const nuri_server_cfg* cfg, nuri_server** out) {
  if (!g || !out) {
    set_error("nuri_server_create: NULL argument");
    return NURI_ERR_INVALID;
  }
  *out = nullptr;
  nuri_server* S = new nuri_server();
  S->g = g;
  S->cfg.slots = cfg && cfg->slots > 0 ? cfg->slots : 4;
  S->cfg.max_batch = cfg && cfg->max_batch > 0 ? cfg->max_batch : 64;
  if (cfg && cfg->mem_budget_bytes > 0) {
    S->cfg.mem_budget_bytes = cfg->mem_budget_bytes;
  } else {  // default: 80 % of the device memory free now
    size_t fr = 0, tot = 0;
    S->cfg.mem_budget_bytes = cudaMemGetInfo(&fr, &tot) == cudaSuccess ? (int64_t)(fr * 0.8)
                                                                      : (8ll << 30);
  }
  // the clique kernels' local memory is reserved by the driver once for the whole context
  // (every stream shares it), so it is charged once against the budget, not per request
  if (g->d.max_out > 64) S->fixed_bytes = clique_local_reserve_bytes();
  for (int i = 0; i < S->cfg.slots; ++i) {
    cudaStream_t st;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
      set_error("nuri_server_create: stream creation failed");
      for (auto x : S->streams) cudaStreamDestroy(x);
      delete S;
      return NURI_ERR_CUDA;
    }
    S->streams.push_back(st);
  }
  for (int i = 0; i < S->cfg.slots; ++i) S->workers.emplace_back(worker_main, S, i);
  *out = S;
  return NURI_OK;
}

nuri_status nuri_server_submit(nuri_server* S, const nuri_request* r, uint64_t* ticket) {
  if (!S || !r || !ticket) {
    set_error("nuri_server_submit: NULL argument");
    return NURI_ERR_INVALID;
  }
  if (r->k < 1 || (r->kind != NURI_REQ_CLIQUES && r->kind != NURI_REQ_ISO)) {
    set_error("nuri_server_submit: bad request kind or k");
    return NURI_ERR_INVALID;
  }
  nuri_server::Req q;
  q.r = *r;
  if (r->kind == NURI_REQ_ISO) {
    const nuri_query& qq = r->query;
    if (qq.nq < 1 || qq.nq > 8 || qq.ne < 0 || !qq.labels || (qq.ne > 0 && (!qq.src || !qq.dst))) {
      set_error("nuri_server_submit: bad query");
      return NURI_ERR_INVALID;
    }
    // a query that cannot run is rejected here, so it never fails a batch it would join
    uint32_t adj[8] = {};
    for (int e = 0; e < qq.ne; ++e) {
      int a = qq.src[e], b = qq.dst[e];
      if (a < 0 || b < 0 || a >= qq.nq || b >= qq.nq || a == b) {
        set_error("nuri_server_submit: bad query edge");
        return NURI_ERR_INVALID;
      }
      adj[a] |= 1u << b;
      adj[b] |= 1u << a;
    }
    uint32_t seen = 1, frontier = 1;
    while (frontier) {
      uint32_t nxt = 0;
      for (int v = 0; v < qq.nq; ++v)
        if ((frontier >> v) & 1) nxt |= adj[v];
      frontier = nxt & ~seen;
      seen |= nxt;
    }
    if (seen != (qq.nq == 32 ? ~0u : ((1u << qq.nq) - 1))) {
      set_error("nuri_server_submit: query is not connected");
      return NURI_ERR_INVALID;
    }
    q.qlab.assign(qq.labels, qq.labels + qq.nq);
    q.qsrc.assign(qq.src, qq.src + qq.ne);
    q.qdst.assign(qq.dst, qq.dst + qq.ne);
  }
  q.mem = request_bytes(S->g, *r);
  q.t_submit = now_ms();
  {
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->stopping) {
      set_error("nuri_server_submit: server is stopping");
      return NURI_ERR_CANCELLED;
    }
    q.ticket = S->next_ticket++;
    *ticket = q.ticket;
    S->live.insert(q.ticket);
    S->pending.push_back(std::move(q));
  }
  S->cv_work.notify_one();
  return NURI_OK;
}

static nuri_status take_done(nuri_server* S, uint64_t ticket, nuri_result** out,
                             nuri_request_times* times) {
  auto it = S->done.find(ticket);
  nuri_server::Done d = it->second;
  S->done.erase(it);
  S->live.erase(ticket);
  *out = d.res;
  if (times) {
    times->queue_ms = d.t_start - d.t_submit;
    times->service_ms = d.t_done - d.t_start;
    times->total_ms = d.t_done - d.t_submit;
    times->start_ms = d.t_start;
    times->done_ms = d.t_done;
    times->mem_bytes = d.mem;
  }
  if (d.status) set_error("%s", d.err.c_str());
  return d.status;
}

nuri_status nuri_server_poll(nuri_server* S, uint64_t ticket, nuri_result** out,
                             nuri_request_times* times) {
  if (!S || !out) {
    set_error("nuri_server_poll: NULL argument");
    return NURI_ERR_INVALID;
  }
  *out = nullptr;
  std::lock_guard<std::mutex> lk(S->mu);
  if (!S->live.count(ticket)) {
    set_error("nuri_server_poll: unknown or already reported ticket");
    return NURI_ERR_INVALID;
  }
  if (!S->done.count(ticket)) return NURI_PENDING;
  return take_done(S, ticket, out, times);
}

nuri_status nuri_server_wait(nuri_server* S, uint64_t ticket, nuri_result** out,
                             nuri_request_times* times) {
  if (!S || !out) {
    set_error("nuri_server_wait: NULL argument");
    return NURI_ERR_INVALID;
  }
  *out = nullptr;
  std::unique_lock<std::mutex> lk(S->mu);
  if (!S->live.count(ticket)) {
    set_error("nuri_server_wait: unknown or already reported ticket");
    return NURI_ERR_INVALID;
  }
  S->cv_done.wait(lk, [&] { return S->done.count(ticket) > 0; });
  return take_done(S, ticket, out, times);
}

nuri_status nuri_server_stats(nuri_server* S, int64_t* batches, int64_t* batched) {
  if (!S) return NURI_ERR_INVALID;
  if (batches) *batches = S->n_batches.load();
  if (batched) *batched = S->n_batched.load();
  return NURI_OK;
}

nuri_status nuri_server_clique_stats(nuri_server* S, int64_t* searches, int64_t* requests) {
  if (!S) return NURI_ERR_INVALID;
  if (searches) *searches = S->n_clique_batches.load();
  if (requests) *requests = S->n_clique_batched.load();
  return NURI_OK;
}

nuri_status nuri_server_budget(nuri_server* S, int64_t* budget_bytes, int64_t* fixed_bytes) {
  if (!S) {
    set_error("nuri_server_budget: NULL server");
    return NURI_ERR_INVALID;
  }
  if (budget_bytes) *budget_bytes = S->cfg.mem_budget_bytes;
  if (fixed_bytes) *fixed_bytes = S->fixed_bytes;
  return NURI_OK;
}

nuri_status nuri_request_bytes(const nuri_graph* g, const nuri_request* r, int64_t* bytes) {
  if (!g || !r || !bytes) {
    set_error("nuri_request_bytes: NULL argument");
    return NURI_ERR_INVALID;
  }
  if (r->k < 1 || (r->kind != NURI_REQ_CLIQUES && r->kind != NURI_REQ_ISO)) {
    set_error("nuri_request_bytes: bad request kind or k");
    return NURI_ERR_INVALID;
  }
  *bytes = request_bytes(g, *r);
  return NURI_OK;
}

void nuri_server_destroy(nuri_server* S) {
  if (!S) return;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stopping = true;
  }
  S->cv_work.notify_all();
  for (auto& t : S->workers) t.join();
  for (auto& kv : S->done)
    if (kv.second.res) nuri_free_result(kv.second.res);
  for (auto st : S->streams) cudaStreamDestroy(st);
  delete S;
}

}  // extern "C"
