// Serving loop with continuous batching: influence queries (select K seeds,
// or the spread of a given seed set) over a resident pool of graphs arrive at
// any time from any thread. A scheduler thread admits them in arrival order
// as soon as a slot (a CUDA stream) is free and the query's workspace fits
// the device-memory budget, so queries that arrive while others are on the
// GPU join them there and their kernels overlap. Workspaces are pooled per
// graph and reused by later queries; the least recently used idle ones are
// freed when a new one would exceed the budget. Results are copied into
// pinned buffers on the query's stream, and an event tells the scheduler the
// query is done. Every query runs the same kernels as its blocking call, so
// its result does not depend on what else is in flight.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "im_common.cuh"

using namespace imgb;

namespace {

double now_s() {
  using namespace std::chrono;
  return duration<double>(steady_clock::now().time_since_epoch()).count();
}

struct Request {
  uint64_t ticket = 0;
  im_request req{};
  std::vector<int32_t> seeds;  // spread: the seed set
  QueryParams q{};
  double t_submit = 0, t_admit = 0, t_done = 0;
  int status = IM_OK;
  std::string detail;  // failed invariant check of an IM_EINTERNAL result
  bool done = false;
  std::vector<int32_t> out_seeds;
  std::vector<uint64_t> out_sigma;
};

struct PooledWs {
  im_workspace *ws = nullptr;
  int32_t graph = 0;
  int32_t R_max = 0;
  size_t bytes = 0;
  bool busy = false;
  uint64_t last_use = 0;
};

struct Slot {
  cudaStream_t stream = nullptr;
  cudaEvent_t done_ev = nullptr;
  int32_t *h_seeds = nullptr;   // pinned: result seeds / staged input seeds
  uint64_t *h_sigma = nullptr;  // pinned: result sigma
  int32_t *h_status = nullptr;  // pinned: device status word
  std::shared_ptr<Request> req;
  PooledWs *pw = nullptr;
};

}  // namespace

struct im_server {
  int device = 0;
  std::vector<const im_graph *> graphs;
  int32_t nmax = 0;
  size_t budget = 0;
  std::vector<Slot> slots;
  std::vector<std::unique_ptr<PooledWs>> pool;
  size_t pool_bytes = 0;                // scheduler thread only; published in stat[]
  uint64_t use_clock = 0;
  std::mutex mu;                       // requests, queue, tickets, stats
  std::condition_variable cv_work;     // scheduler: new submissions
  std::condition_variable cv_done;     // waiters: completions
  std::deque<std::shared_ptr<Request>> queue;
  std::map<uint64_t, std::shared_ptr<Request>> tickets;
  uint64_t next_ticket = 1;
  bool stop = false;
  int init_status = IM_OK;
  std::thread worker;
  int64_t stat[IM_SERVER_STAT_COUNT] = {0};
  double t0 = 0;
};

namespace {

void finish(im_server *sv, Slot &sl, int status) {
  std::shared_ptr<Request> r = sl.req;
  const bool select = r->req.kind == IM_REQUEST_SELECT;
  if (status == IM_OK && *sl.h_status != 0) status = *sl.h_status;
  std::string detail;
  if (status == IM_EINTERNAL) detail = api_check_text(sl.pw->ws, sl.stream);
  if (status == IM_OK) {
    if (select) {
      r->out_seeds.assign(sl.h_seeds, sl.h_seeds + r->req.K);
      r->out_sigma.assign(sl.h_sigma, sl.h_sigma + r->req.K);
    } else {
      r->out_sigma.assign(sl.h_sigma, sl.h_sigma + 1);
    }
  }
  sl.pw->busy = false;
  sl.pw->last_use = ++sv->use_clock;
  sl.pw = nullptr;
  sl.req.reset();
  std::lock_guard<std::mutex> lock(sv->mu);
  r->status = status;
  r->detail = std::move(detail);
  r->t_done = now_s() - sv->t0;
  r->done = true;
  ++sv->stat[IM_SERVER_STAT_COMPLETED];
  --sv->stat[IM_SERVER_STAT_IN_FLIGHT];
  sv->cv_done.notify_all();
}

// A pooled workspace for graph g with R_max >= R that is idle, or a new one
// within the budget (idle ones are freed oldest-use first to make room).
// Returns nullptr when the request has to wait for running queries.
PooledWs *acquire_ws(im_server *sv, int32_t gi, int32_t R, int *err) {
  PooledWs *best = nullptr;
  for (auto &p : sv->pool)
    if (!p->busy && p->graph == gi && p->R_max >= R && (!best || p->R_max < best->R_max))
      best = p.get();
  if (best) return best;
  const im_graph *g = sv->graphs[gi];
  const size_t need = api_ws_bytes(g, R);
  while (sv->pool_bytes + need > sv->budget) {
    PooledWs *victim = nullptr;
    for (auto &p : sv->pool)
      if (!p->busy && (!victim || p->last_use < victim->last_use)) victim = p.get();
    if (!victim) return nullptr;  // everything is in use: wait
    api_ws_destroy(victim->ws);
    sv->pool_bytes -= victim->bytes;
    {
      std::lock_guard<std::mutex> lock(sv->mu);
      ++sv->stat[IM_SERVER_STAT_WS_EVICTED];
      sv->stat[IM_SERVER_STAT_POOL_BYTES] = (int64_t)sv->pool_bytes;
    }
    sv->pool.erase(std::find_if(sv->pool.begin(), sv->pool.end(),
                                [&](const std::unique_ptr<PooledWs> &p) { return p.get() == victim; }));
  }
  im_workspace *ws = nullptr;
  int rc = api_ws_create(g, R, &ws);
  if (rc == IM_OK) rc = api_ws_seed_capacity(ws, g->n);
  if (rc != IM_OK) {
    if (ws) api_ws_destroy(ws);
    *err = rc;
    return nullptr;
  }
  auto p = std::make_unique<PooledWs>();
  p->ws = ws;
  p->graph = gi;
  p->R_max = R;
  p->bytes = need;
  sv->pool_bytes += need;
  {
    std::lock_guard<std::mutex> lock(sv->mu);
    ++sv->stat[IM_SERVER_STAT_WS_CREATED];
    sv->stat[IM_SERVER_STAT_POOL_BYTES] = (int64_t)sv->pool_bytes;
    if ((int64_t)sv->pool_bytes > sv->stat[IM_SERVER_STAT_POOL_BYTES_PEAK])
      sv->stat[IM_SERVER_STAT_POOL_BYTES_PEAK] = (int64_t)sv->pool_bytes;
  }
  sv->pool.push_back(std::move(p));
  return sv->pool.back().get();
}

// Queue the query's kernels, result copies and completion event on its slot.
int launch(im_server *sv, Slot &sl) {
  Request &r = *sl.req;
  const im_graph *g = sv->graphs[r.req.graph];
  im_workspace *ws = sl.pw->ws;
  cudaStream_t s = sl.stream;
  cudaError_t e = cudaMemsetAsync(ws->d_status, 0, sizeof(int32_t), s);
  if (e != cudaSuccess) return api_cuda_error(e, "status reset");
  int rc;
  if (r.req.kind == IM_REQUEST_SELECT) {
    rc = api_enqueue_select(g, ws, r.req.K, r.q, ws->d_seeds_out, ws->d_sigma_out, s);
    if (rc != IM_OK) return rc;
    e = cudaMemcpyAsync(sl.h_seeds, ws->d_seeds_out, sizeof(int32_t) * r.req.K,
                        cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(sl.h_sigma, ws->d_sigma_out, sizeof(uint64_t) * r.req.K,
                          cudaMemcpyDeviceToHost, s);
  } else {
    if (!r.seeds.empty()) {
      std::memcpy(sl.h_seeds, r.seeds.data(), sizeof(int32_t) * r.seeds.size());
      e = cudaMemcpyAsync(ws->d_seeds_in, sl.h_seeds, sizeof(int32_t) * r.seeds.size(),
                          cudaMemcpyHostToDevice, s);
      if (e != cudaSuccess) return api_cuda_error(e, "seed copy");
    }
    rc = api_enqueue_spread(g, ws, ws->d_seeds_in, (int32_t)r.seeds.size(), r.q,
                            ws->d_sigma_out, s);
    if (rc != IM_OK) return rc;
    e = cudaMemcpyAsync(sl.h_sigma, ws->d_sigma_out, sizeof(uint64_t), cudaMemcpyDeviceToHost, s);
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(sl.h_status, ws->d_status, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaEventRecord(sl.done_ev, s);
  if (e != cudaSuccess) return api_cuda_error(e, "result copies");
  return IM_OK;
}

void scheduler(im_server *sv) {
  cudaSetDevice(sv->device);
  for (;;) {
    bool progress = false;
    // completions
    for (Slot &sl : sv->slots) {
      if (!sl.req) continue;
      const cudaError_t e = cudaEventQuery(sl.done_ev);
      if (e == cudaErrorNotReady) continue;
      finish(sv, sl, e == cudaSuccess ? IM_OK : api_cuda_error(e, "query on the device"));
      progress = true;
    }
    // admissions, in arrival order
    for (;;) {
      Slot *free_slot = nullptr;
      for (Slot &sl : sv->slots)
        if (!sl.req) {
          free_slot = &sl;
          break;
        }
      if (!free_slot) break;
      std::shared_ptr<Request> r;
      {
        std::lock_guard<std::mutex> lock(sv->mu);
        if (sv->queue.empty()) break;
        r = sv->queue.front();
      }
      int err = IM_OK;
      PooledWs *pw = acquire_ws(sv, r->req.graph, r->req.R, &err);
      if (!pw && err == IM_OK) break;  // wait until running queries give memory back
      {
        std::lock_guard<std::mutex> lock(sv->mu);
        sv->queue.pop_front();
        r->t_admit = now_s() - sv->t0;
        ++sv->stat[IM_SERVER_STAT_ADMITTED];
        ++sv->stat[IM_SERVER_STAT_IN_FLIGHT];
        if (sv->stat[IM_SERVER_STAT_IN_FLIGHT] > sv->stat[IM_SERVER_STAT_IN_FLIGHT_PEAK])
          sv->stat[IM_SERVER_STAT_IN_FLIGHT_PEAK] = sv->stat[IM_SERVER_STAT_IN_FLIGHT];
      }
      free_slot->req = r;
      if (!pw) {
        free_slot->pw = nullptr;
        std::lock_guard<std::mutex> lock(sv->mu);
        r->status = err;
        r->t_done = now_s() - sv->t0;
        r->done = true;
        free_slot->req.reset();
        ++sv->stat[IM_SERVER_STAT_COMPLETED];
        --sv->stat[IM_SERVER_STAT_IN_FLIGHT];
        sv->cv_done.notify_all();
        continue;
      }
      pw->busy = true;
      free_slot->pw = pw;
      const int rc = launch(sv, *free_slot);
      if (rc != IM_OK) {
        cudaStreamSynchronize(free_slot->stream);
        finish(sv, *free_slot, rc);
      }
      progress = true;
    }
    std::unique_lock<std::mutex> lock(sv->mu);
    bool busy = false;
    for (Slot &sl : sv->slots) busy = busy || (bool)sl.req;
    if (sv->stop && sv->queue.empty() && !busy) break;
    if (!progress) {
      // new work wakes the scheduler; running queries are polled every 20 us
      sv->cv_work.wait_for(lock, std::chrono::microseconds(busy ? 20 : 2000));
    }
  }
}

void server_free(im_server *sv) {
  for (Slot &sl : sv->slots) {
    if (sl.stream) cudaStreamDestroy(sl.stream);
    if (sl.done_ev) cudaEventDestroy(sl.done_ev);
    if (sl.h_seeds) cudaFreeHost(sl.h_seeds);
    if (sl.h_sigma) cudaFreeHost(sl.h_sigma);
    if (sl.h_status) cudaFreeHost(sl.h_status);
  }
  for (auto &p : sv->pool) api_ws_destroy(p->ws);
  sv->pool.clear();
}

}  // namespace

extern "C" {

int im_server_create(const im_graph *const *graphs, int32_t num_graphs, int32_t slots,
                     int64_t memory_budget, im_server **out) {
  if (!graphs || !out || num_graphs < 1 || slots < 1 || slots > 256 || memory_budget < 1)
    return api_error(IM_EINVAL, "bad server arguments");
  im_server *sv = new (std::nothrow) im_server();
  if (!sv) return api_error(IM_ENOMEM, "host allocation failed");
  sv->graphs.assign(graphs, graphs + num_graphs);
  for (int32_t i = 0; i < num_graphs; ++i) {
    if (!graphs[i] || graphs[i]->device != graphs[0]->device) {
      delete sv;
      return api_error(IM_EINVAL, "graph %d missing or on another device", i);
    }
    sv->nmax = std::max(sv->nmax, graphs[i]->n);
  }
  sv->device = graphs[0]->device;
  sv->budget = (size_t)memory_budget;
  sv->t0 = now_s();
  DeviceGuard dg(sv->device);
  sv->slots.resize(slots);
  cudaError_t e = cudaSuccess;
  for (Slot &sl : sv->slots) {
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.done_ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaHostAlloc(reinterpret_cast<void **>(&sl.h_seeds), 4 * (size_t)sv->nmax, 0);
    if (e == cudaSuccess) e = cudaHostAlloc(reinterpret_cast<void **>(&sl.h_sigma), 8 * (size_t)sv->nmax, 0);
    if (e == cudaSuccess) e = cudaHostAlloc(reinterpret_cast<void **>(&sl.h_status), 4, 0);
  }
  if (e != cudaSuccess) {
    server_free(sv);
    delete sv;
    return api_cuda_error(e, "server slots");
  }
  sv->worker = std::thread(scheduler, sv);
  *out = sv;
  return IM_OK;
}

int im_server_submit(im_server *sv, const im_request *r, uint64_t *ticket) {
  if (!sv || !r || !ticket) return api_error(IM_EINVAL, "null argument");
  if (r->graph < 0 || r->graph >= (int32_t)sv->graphs.size())
    return api_error(IM_EINVAL, "graph index %d outside the server's pool", r->graph);
  const im_graph *g = sv->graphs[r->graph];
  if (r->kind != IM_REQUEST_SELECT && r->kind != IM_REQUEST_SPREAD)
    return api_error(IM_EINVAL, "unknown request kind %d", r->kind);
  if (r->flags & IM_ALGO_FUSED_SAMPLING)
    return api_error(IM_EINVAL, "IM_ALGO_FUSED_SAMPLING is not served");
  auto req = std::make_shared<Request>();
  int rc = api_query_params(g, r->R, r->p, r->rng_seed, r->flags, &req->q);
  if (rc != IM_OK) return rc;
  if (r->kind == IM_REQUEST_SELECT) {
    if (r->K < 1 || r->K > g->n) return api_error(IM_EINVAL, "K=%d outside [1, n=%d]", r->K, g->n);
  } else {
    if (r->K < 0 || r->K > g->n || (r->K > 0 && !r->seeds))
      return api_error(IM_EINVAL, "spread: %d seeds (at most n, host array)", r->K);
    for (int32_t i = 0; i < r->K; ++i)
      if (r->seeds[i] < 0 || r->seeds[i] >= g->n)
        return api_error(IM_EINVAL, "seed id %d out of range", r->seeds[i]);
    req->seeds.assign(r->seeds, r->seeds + r->K);
  }
  if (api_ws_bytes(g, r->R) > sv->budget)
    return api_error(IM_ENOMEM, "the query's workspace (%zu bytes) exceeds the memory budget",
                     api_ws_bytes(g, r->R));
  req->req = *r;
  req->req.seeds = nullptr;
  std::lock_guard<std::mutex> lock(sv->mu);
  if (sv->stop) return api_error(IM_EBUSY, "server is shutting down");
  req->ticket = sv->next_ticket++;
  req->t_submit = now_s() - sv->t0;
  sv->queue.push_back(req);
  sv->tickets[req->ticket] = req;
  ++sv->stat[IM_SERVER_STAT_SUBMITTED];
  if ((int64_t)sv->queue.size() > sv->stat[IM_SERVER_STAT_QUEUE_PEAK])
    sv->stat[IM_SERVER_STAT_QUEUE_PEAK] = (int64_t)sv->queue.size();
  sv->cv_work.notify_one();
  *ticket = req->ticket;
  return IM_OK;
}

int im_server_wait(im_server *sv, uint64_t ticket, int64_t timeout_us, int32_t *out_seeds,
                   uint64_t *out_sigma_R, double *out_times) {
  if (!sv) return api_error(IM_EINVAL, "null server");
  std::unique_lock<std::mutex> lock(sv->mu);
  auto it = sv->tickets.find(ticket);
  if (it == sv->tickets.end()) return api_error(IM_EINVAL, "unknown ticket %llu", (unsigned long long)ticket);
  std::shared_ptr<Request> r = it->second;
  if (!r->done) {
    if (timeout_us > 0)
      sv->cv_done.wait_for(lock, std::chrono::microseconds(timeout_us), [&] { return r->done; });
    else if (timeout_us < 0)
      sv->cv_done.wait(lock, [&] { return r->done; });
  }
  if (!r->done) return api_error(IM_EBUSY, "query %llu still running", (unsigned long long)ticket);
  sv->tickets.erase(it);
  if (out_times) {
    out_times[0] = r->t_submit;
    out_times[1] = r->t_admit;
    out_times[2] = r->t_done;
  }
  if (r->status != IM_OK)
    return api_error(r->status, "query %llu failed on the device%s%s", (unsigned long long)ticket,
                     r->detail.empty() ? "" : ": ", r->detail.c_str());
  if (r->req.kind == IM_REQUEST_SELECT) {
    if (out_seeds) std::memcpy(out_seeds, r->out_seeds.data(), sizeof(int32_t) * r->out_seeds.size());
    if (out_sigma_R) std::memcpy(out_sigma_R, r->out_sigma.data(), sizeof(uint64_t) * r->out_sigma.size());
  } else if (out_sigma_R) {
    out_sigma_R[0] = r->out_sigma[0];
  }
  return IM_OK;
}

int im_server_stats(im_server *sv, int64_t *out) {
  if (!sv || !out) return api_error(IM_EINVAL, "null argument");
  std::lock_guard<std::mutex> lock(sv->mu);
  for (int i = 0; i < IM_SERVER_STAT_COUNT; ++i) out[i] = sv->stat[i];
  out[IM_SERVER_STAT_QUEUED] = (int64_t)sv->queue.size();
  out[IM_SERVER_STAT_BUDGET] = (int64_t)sv->budget;
  return IM_OK;
}

int im_server_destroy(im_server *sv) {
  if (!sv) return api_error(IM_EINVAL, "null server");
  {
    std::lock_guard<std::mutex> lock(sv->mu);
    sv->stop = true;
    sv->cv_work.notify_all();
  }
  if (sv->worker.joinable()) sv->worker.join();  // drains queued and running queries
  DeviceGuard dg(sv->device);
  server_free(sv);
  delete sv;
  return IM_OK;
}

}  // extern "C"
