// Serving loop over one resident graph: single-source requests (SSSP, BFS or
// PPR) arrive one at a time and are run by the buffered engine in batches.
//
// Continuous batching: the server owns `lanes` independent batch slots, each
// with its own stream, engine workspace and output rows. fg_server_poll
// launches the waiting requests of one kind on every free lane (the kind whose
// oldest request has waited longest) and reports the requests whose batch has
// completed. Lanes launch on 1/lanes of the GPU's resident grid by default, so
// batches of different kinds and ages run on the device at the same time. A
// lane becomes free again once every request of its batch has been released:
// the memory the server holds is fixed at creation (lanes x max_batch rows),
// which is how requests are admitted by HBM budget.
#include <algorithm>
#include <chrono>
#include <cstring>
#include <deque>
#include <mutex>
#include <unordered_map>
#include <vector>

#include "fg_host.h"

using namespace fg;

namespace {

int64_t now_ns() {
  return std::chrono::duration_cast<std::chrono::nanoseconds>(std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

struct Request {
  int32_t kind = 0, source = 0;
  int32_t status = FG_OK;
  int32_t lane = -1, row = -1, batch = 0;
  int64_t submit_ns = 0, launch_ns = 0, done_ns = 0;
  bool done = false;
};

struct Lane {
  Workspace ws;
  cudaStream_t stream = nullptr;
  cudaEvent_t done_ev = nullptr;
  DevBuf src, out, out_r, mass;  // device: sources, rows (u32 or f32), PPR residual rows, PPR mass
  int32_t *h_src = nullptr;      // pinned staging of the batch's sources
  double *h_mass = nullptr;      // pinned copy of the batch's PPR mass
  int kind = -1;
  std::vector<uint64_t> reqs;    // requests of the batch in flight or awaiting release
  int live = 0;                  // requests not yet released
  bool running = false;          // launched, completion not yet observed
};

}  // namespace

struct fg_server {
  fg_graph *g = nullptr;
  fg_server_opts o{};
  int device = 0;
  std::vector<Lane> lanes;
  std::mutex mu;
  std::deque<uint64_t> queue[3];           // waiting requests per kind, oldest first
  std::unordered_map<uint64_t, Request> reqs;
  std::deque<uint64_t> finished;           // completed, not yet reported by poll
  uint64_t next_id = 1;
};

extern "C" void fg_default_server_opts(fg_server_opts *o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->struct_size = sizeof(fg_server_opts);
  o->lanes = 4;
  o->max_batch = 256;
  o->full_grid = 0;
  o->alpha = 0.15f;
  o->eps = 1e-6f;
  o->hbm_budget = 0;
  for (int k = 0; k < 3; ++k) fg_default_opts(&o->opts[k]);
}

namespace {

// Device bytes one request of the given kind holds while its batch is in
// flight: output rows plus the engine's per-query state and buffers.
double per_request_bytes(const fg_graph *g, int kind) {
  const double n = (double)g->n, keys = (double)g->nparts * 36.0 + n / 8.0;
  const bool relabelled = g->dg.orig != nullptr;
  if (kind == FG_QUERY_PPR) return 8.0 * n + (relabelled ? 12.0 : 4.0) * n + keys;
  return 4.0 * n + (relabelled ? 4.0 : 0.0) * n + keys;
}

fg_status launch_lane(fg_server *s, Lane &L, int kind) {
  fg_graph *g = s->g;
  const int64_t n = g->n;
  std::deque<uint64_t> &q = s->queue[kind];
  const int nb = (int)std::min<size_t>(q.size(), (size_t)s->o.max_batch);
  L.reqs.clear();
  const int64_t t = now_ns();
  for (int i = 0; i < nb; ++i) {
    const uint64_t id = q.front();
    q.pop_front();
    Request &r = s->reqs[id];
    r.lane = (int)(&L - s->lanes.data());
    r.row = i;
    r.batch = nb;
    r.launch_ns = t;
    L.h_src[i] = r.source;
    L.reqs.push_back(id);
  }
  L.kind = kind;
  L.live = nb;
  L.running = true;
  CUDA_TRY(cudaMemcpyAsync(L.src.p, L.h_src, 4 * (size_t)nb, cudaMemcpyHostToDevice, L.stream));
  const fg_opts *o = &s->o.opts[kind];
  const int div = s->o.full_grid ? 1 : s->o.lanes;
  fg_status st;
  if (kind == FG_QUERY_PPR) {
    st = run_batch_on(g, L.ws, false, div, Q_PPR, L.src.as<int32_t>(), nb, nullptr, s->o.alpha, s->o.eps,
                      L.out.as<float>(), L.out_r.as<float>(), L.mass.as<double>(), L.stream, o);
    if (st == FG_OK)
      CUDA_TRY(cudaMemcpyAsync(L.h_mass, L.mass.p, 8 * (size_t)nb, cudaMemcpyDeviceToHost, L.stream));
  } else {
    st = run_batch_on(g, L.ws, false, div, kind == FG_QUERY_BFS ? Q_BFS : Q_SSSP, L.src.as<int32_t>(), nb,
                      L.out.as<uint32_t>(), 0.f, 0.f, nullptr, nullptr, nullptr, L.stream, o);
  }
  (void)n;
  if (st != FG_OK) return st;
  CUDA_TRY(cudaEventRecord(L.done_ev, L.stream));
  return FG_OK;
}

}  // namespace

extern "C" fg_status fg_server_create(fg_graph *g, const fg_server_opts *opts, fg_server **out) {
  if (!g || !out) return fail(FG_ERR_INVALID_ARG, "NULL argument");
  *out = nullptr;
  fg_server_opts o;
  fg_default_server_opts(&o);
  if (opts) {
    const size_t sz = std::min<size_t>(opts->struct_size, sizeof(fg_server_opts));
    if (sz > sizeof(uint32_t))
      std::memcpy(reinterpret_cast<char *>(&o) + sizeof(uint32_t), reinterpret_cast<const char *>(opts) + sizeof(uint32_t),
                  sz - sizeof(uint32_t));
    o.struct_size = sizeof(fg_server_opts);
    for (int k = 0; k < 3; ++k)
      if (o.opts[k].struct_size == 0) fg_default_opts(&o.opts[k]);
  }
  if (o.lanes < 1 || o.lanes > 64) return fail(FG_ERR_INVALID_ARG, "lanes must be in [1, 64]");
  if (o.max_batch < 1) return fail(FG_ERR_INVALID_ARG, "max_batch must be >= 1");
  if (!(o.alpha > 0.f && o.alpha < 1.f)) return fail(FG_ERR_INVALID_ARG, "alpha must be in (0, 1)");
  if (!(o.eps > 0.f)) return fail(FG_ERR_INVALID_ARG, "eps must be > 0");
  if (o.hbm_budget < 0) return fail(FG_ERR_INVALID_ARG, "hbm_budget must be >= 0");
  CUDA_TRY(cudaSetDevice(g->device));
  // admission by HBM budget: every lane must be able to hold a full batch of
  // the most expensive kind
  int64_t budget = o.hbm_budget;
  if (budget == 0) {
    size_t fr = 0, tot = 0;
    CUDA_TRY(cudaMemGetInfo(&fr, &tot));
    budget = (int64_t)(0.6 * (double)fr);
  }
  const double per_q = std::max(per_request_bytes(g, FG_QUERY_PPR), per_request_bytes(g, FG_QUERY_SSSP));
  const int64_t fit = (int64_t)((double)budget / ((double)o.lanes * per_q));
  if (fit < 1) return fail(FG_ERR_OOM, "HBM budget %lld B holds no batch of one request per lane", (long long)budget);
  o.max_batch = (int32_t)std::min<int64_t>(o.max_batch, fit);

  fg_server *s = new fg_server;
  s->g = g;
  s->o = o;
  s->device = g->device;
  s->lanes.resize((size_t)o.lanes);
  const size_t rows = (size_t)o.max_batch * (size_t)g->n;
  fg_status st = FG_OK;
  for (Lane &L : s->lanes) {
    cudaError_t e = cudaStreamCreateWithFlags(&L.stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&L.done_ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = L.src.reserve(4 * (size_t)o.max_batch);
    if (e == cudaSuccess) e = L.out.reserve(4 * rows);
    if (e == cudaSuccess) e = L.out_r.reserve(4 * rows);
    if (e == cudaSuccess) e = L.mass.reserve(8 * (size_t)o.max_batch);
    if (e == cudaSuccess) e = cudaMallocHost(&L.h_src, 4 * (size_t)o.max_batch);
    if (e == cudaSuccess) e = cudaMallocHost(&L.h_mass, 8 * (size_t)o.max_batch);
    if (e != cudaSuccess) {
      st = fail(e == cudaErrorMemoryAllocation ? FG_ERR_OOM : FG_ERR_CUDA, "server lane: %s", cudaGetErrorString(e));
      break;
    }
  }
  if (st != FG_OK) {
    fg_server_destroy(s);
    return st;
  }
  *out = s;
  return FG_OK;
}

extern "C" fg_status fg_server_destroy(fg_server *s) {
  if (!s) return FG_OK;
  cudaSetDevice(s->device);
  for (Lane &L : s->lanes) {
    if (L.stream) {
      fg_sync(L.stream);  // wait for the lane and collect its status slot
      cudaStreamDestroy(L.stream);
    }
    if (L.done_ev) cudaEventDestroy(L.done_ev);
    L.ws.release_all();
    L.src.release();
    L.out.release();
    L.out_r.release();
    L.mass.release();
    if (L.h_src) cudaFreeHost(L.h_src);
    if (L.h_mass) cudaFreeHost(L.h_mass);
  }
  delete s;
  return FG_OK;
}

extern "C" fg_status fg_server_submit(fg_server *s, int32_t kind, int32_t source, uint64_t *id) {
  if (!s || !id) return fail(FG_ERR_INVALID_ARG, "NULL argument");
  if (kind < FG_QUERY_SSSP || kind > FG_QUERY_PPR) return fail(FG_ERR_INVALID_ARG, "unknown query kind %d", kind);
  if (source < 0 || source >= s->g->n) return fail(FG_ERR_INVALID_ARG, "source %d out of range", source);
  std::lock_guard<std::mutex> lk(s->mu);
  const uint64_t i = s->next_id++;
  Request &r = s->reqs[i];
  r.kind = kind;
  r.source = source;
  r.submit_ns = now_ns();
  s->queue[kind].push_back(i);
  *id = i;
  return FG_OK;
}

extern "C" fg_status fg_server_poll(fg_server *s, uint64_t *done, int32_t cap, int32_t *n_done) {
  if (!s || !n_done || cap < 0 || (cap > 0 && !done)) return fail(FG_ERR_INVALID_ARG, "bad poll arguments");
  std::lock_guard<std::mutex> lk(s->mu);
  CUDA_TRY(cudaSetDevice(s->device));
  fg_status first = FG_OK;
  // 1. batches that have completed
  for (Lane &L : s->lanes) {
    if (!L.running) continue;
    const cudaError_t q = cudaEventQuery(L.done_ev);
    if (q == cudaErrorNotReady) continue;
    L.running = false;
    fg_status st = fg_sync(L.stream);  // collects the batch's device status
    if (q != cudaSuccess && st == FG_OK) st = fail(FG_ERR_CUDA, "%s", cudaGetErrorString(q));
    if (st != FG_OK && first == FG_OK) first = st;
    const int64_t t = now_ns();
    for (uint64_t id : L.reqs) {
      Request &r = s->reqs[id];
      r.done = true;
      r.done_ns = t;
      r.status = st;
      s->finished.push_back(id);
    }
  }
  // 2. free lanes take the waiting requests of the kind that has waited longest
  for (Lane &L : s->lanes) {
    if (L.running || L.live > 0) continue;
    int kind = -1;
    int64_t oldest = 0;
    for (int k = 0; k < 3; ++k) {
      if (s->queue[k].empty()) continue;
      const int64_t t = s->reqs[s->queue[k].front()].submit_ns;
      if (kind < 0 || t < oldest) {
        kind = k;
        oldest = t;
      }
    }
    if (kind < 0) break;
    fg_status st = launch_lane(s, L, kind);
    if (st != FG_OK) {
      // the batch never ran: its requests complete with the launch error
      L.running = false;
      const int64_t t = now_ns();
      for (uint64_t id : L.reqs) {
        Request &r = s->reqs[id];
        r.done = true;
        r.done_ns = t;
        r.status = st;
        s->finished.push_back(id);
      }
      if (first == FG_OK) first = st;
    }
  }
  int32_t k = 0;
  while (k < cap && !s->finished.empty()) {
    done[k++] = s->finished.front();
    s->finished.pop_front();
  }
  *n_done = k;
  return first;
}

extern "C" fg_status fg_server_info(fg_server *s, uint64_t id, fg_request_info *info) {
  if (!s || !info) return fail(FG_ERR_INVALID_ARG, "NULL argument");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(id);
  if (it == s->reqs.end()) return fail(FG_ERR_INVALID_ARG, "unknown request %llu", (unsigned long long)id);
  const Request &r = it->second;
  std::memset(info, 0, sizeof(*info));
  info->kind = r.kind;
  info->source = r.source;
  info->status = r.done ? r.status : -1;
  info->batch_size = r.batch;
  info->submit_ns = r.submit_ns;
  info->launch_ns = r.launch_ns;
  info->done_ns = r.done_ns;
  if (r.done && r.lane >= 0) {
    Lane &L = s->lanes[(size_t)r.lane];
    const size_t off = (size_t)r.row * (size_t)s->g->n;
    if (r.kind == FG_QUERY_PPR) {
      info->result = L.out.as<float>() + off;
      info->residual = L.out_r.as<float>() + off;
      info->mass = L.h_mass[r.row];
    } else {
      info->result = L.out.as<uint32_t>() + off;
    }
  }
  return FG_OK;
}

extern "C" fg_status fg_server_release(fg_server *s, uint64_t id) {
  if (!s) return fail(FG_ERR_INVALID_ARG, "NULL argument");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(id);
  if (it == s->reqs.end()) return fail(FG_ERR_INVALID_ARG, "unknown request %llu", (unsigned long long)id);
  if (!it->second.done) return fail(FG_ERR_INVALID_ARG, "request %llu has not completed", (unsigned long long)id);
  const int lane = it->second.lane;
  s->reqs.erase(it);
  if (lane >= 0) s->lanes[(size_t)lane].live -= 1;
  return FG_OK;
}
