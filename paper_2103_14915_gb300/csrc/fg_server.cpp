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
//
// Slot-level batching (opts.continuous): SSSP and BFS requests instead join a
// running launch of the group engine one query lane at a time. Each of the two
// kinds has a slot lane: a fixed set of query lanes (slots) with their state,
// a result row per slot, and a mailbox in mapped host memory. The host writes
// a request's source and a new sequence number into a free slot; the launch
// picks it up at its next round boundary, and when the lane's query has no
// pending work left it copies the row out and posts the sequence number back,
// so a request neither waits for a batch to fill nor for the slowest query of
// its batch. A launch ends once it holds no query and finds no new request;
// poll starts a new one when a request waits in the mailbox.
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
  int32_t slot = -1;  // slot of the kind's slot lane (slot-level batching), else -1
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

// Slot lane of one kind (SSSP or BFS) under slot-level batching.
struct SlotLane {
  int kind = -1, qtype = 0;
  int G = 32, glog2 = 5, ngroups = 0, nslots = 0, blocks = 0, gi = 2;
  cudaStream_t stream = nullptr;
  cudaEvent_t done_ev = nullptr;
  DevBuf D, pend, dirty, items, res, occ, seen, gact, ctrl, reach, lstart;
  ServeBox *box = nullptr;        // mapped host memory (host address)
  ServeBox *box_dev = nullptr;    // its device address
  Ctrl *h_ctrl = nullptr;         // pinned copy of the control block after each launch
  std::vector<uint64_t> slot_req;  // request in each slot (0 = free)
  std::vector<uint32_t> slot_seq;  // last sequence number written to each slot
  std::vector<uint8_t> slot_done;  // the slot's request has completed
  uint32_t round0 = 0;             // first round of the next launch (a launch yields after max_rounds)
  bool running = false, need_init = true;
  void release_all() {
    DevBuf *all[] = {&D, &pend, &dirty, &items, &res, &occ, &seen, &gact, &ctrl, &reach, &lstart};
    for (DevBuf *b : all) b->release();
    if (box) cudaFreeHost(box);
    if (h_ctrl) cudaFreeHost(h_ctrl);
    if (done_ev) cudaEventDestroy(done_ev);
    if (stream) cudaStreamDestroy(stream);
    box = box_dev = nullptr;
    h_ctrl = nullptr;
    done_ev = nullptr;
    stream = nullptr;
  }
};

}  // namespace

struct fg_server {
  fg_graph *g = nullptr;
  fg_server_opts o{};
  int device = 0;
  std::vector<Lane> lanes;
  SlotLane slot_lanes[2];                  // slot-level batching: SSSP, BFS
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
  o->continuous = 0;
  o->slots = 128;
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

// Device bytes of one slot of a slot lane with groups of G: its share of the
// vertex-major state, pending masks, dirty flags and work items, and its row.
double per_slot_bytes(const fg_graph *g, int G) {
  const double npad = (double)g->nparts * (double)g->S;
  return 4.0 * npad + (12.0 * npad + 24.0 * (double)g->nparts + 16.0 * (double)g->hub_chunks + 8.0) / (double)G +
         4.0 * (double)g->n;
}

fg_status create_slot_lane(fg_server *s, SlotLane &C, int kind, int nslots, int G, int div) {
  fg_graph *g = s->g;
  C.kind = kind;
  C.qtype = kind == FG_QUERY_BFS ? Q_BFS : Q_SSSP;
  C.G = G;
  C.glog2 = G == 8 ? 3 : (G == 16 ? 4 : 5);
  C.gi = C.glog2 - 3;
  C.ngroups = nslots / G;
  C.nslots = nslots;
  if (!group_fits(g->S, G))
    return fail(FG_ERR_UNSUPPORTED, "group %d does not fit shared memory with partitions of %d vertices", G, g->S);
  if (g->group_blocks[C.gi] == 0)
    CUDA_TRY(group_grid_size(g->S, G, &g->group_blocks[C.gi], &g->group_threads[C.gi], &g->group_smem[C.gi]));
  C.blocks = div > 1 ? std::max(1, g->group_blocks[C.gi] / div) : g->group_blocks[C.gi];
  const size_t npad = (size_t)g->nparts * (size_t)g->S, ng = (size_t)C.ngroups;
  const uint64_t hub_cap = (uint64_t)ng * g->hub_chunks;
  if (hub_cap + (uint64_t)ng * (uint64_t)g->nparts >= 0xFFFFFFFFull)
    return fail(FG_ERR_UNSUPPORTED, "too many work items for one slot lane; lower slots");
  CUDA_TRY(cudaStreamCreateWithFlags(&C.stream, cudaStreamNonBlocking));
  CUDA_TRY(cudaEventCreateWithFlags(&C.done_ev, cudaEventDisableTiming));
  CUDA_TRY(C.D.reserve(4 * ng * npad * (size_t)G));
  CUDA_TRY(C.pend.reserve(8 * ng * npad));
  CUDA_TRY(C.dirty.reserve(8 * ng * (size_t)g->nparts));
  CUDA_TRY(C.items.reserve(16 * (size_t)(hub_cap + (uint64_t)ng * (uint64_t)g->nparts)));
  CUDA_TRY(C.res.reserve(4 * (size_t)nslots * (size_t)g->n));
  CUDA_TRY(C.occ.reserve(4 * ng));
  CUDA_TRY(C.seen.reserve(4 * (size_t)nslots));
  CUDA_TRY(C.gact.reserve(8 * ng));
  if (C.qtype == Q_BFS) {
    CUDA_TRY(C.reach.reserve(4 * ng * npad));
    CUDA_TRY(C.lstart.reserve(4 * (size_t)nslots));
  }
  CUDA_TRY(C.ctrl.reserve(sizeof(Ctrl)));
  const size_t box_bytes = sizeof(ServeBox) + sizeof(ServeSlot) * (size_t)(nslots - 1);
  void *hb = nullptr;
  CUDA_TRY(cudaHostAlloc(&hb, box_bytes, cudaHostAllocMapped));
  std::memset(hb, 0, box_bytes);
  C.box = reinterpret_cast<ServeBox *>(hb);
  void *db = nullptr;
  CUDA_TRY(cudaHostGetDevicePointer(&db, hb, 0));
  C.box_dev = reinterpret_cast<ServeBox *>(db);
  CUDA_TRY(cudaMallocHost(&C.h_ctrl, sizeof(Ctrl)));
  std::memset(C.h_ctrl, 0, sizeof(Ctrl));
  C.slot_req.assign((size_t)nslots, 0);
  C.slot_seq.assign((size_t)nslots, 0);
  C.slot_done.assign((size_t)nslots, 0);
  C.need_init = true;
  return FG_OK;
}

// Starts a launch on the slot lane; with need_init it first clears the lane
// state the kernel keeps between launches (occupancy, sequence numbers seen).
fg_status launch_slot_lane(fg_server *s, SlotLane &C) {
  fg_graph *g = s->g;
  const fg_opts &o = s->o.opts[C.kind];
  if (C.need_init) {
    CUDA_TRY(cudaMemsetAsync(C.occ.p, 0, C.occ.bytes, C.stream));
    CUDA_TRY(cudaMemsetAsync(C.seen.p, 0, C.seen.bytes, C.stream));
  }
  CUDA_TRY(cudaMemsetAsync(C.ctrl.p, 0, sizeof(Ctrl), C.stream));
  GroupArgs a;
  a.g = g->dg;
  a.qtype = C.qtype;
  a.nq = C.nslots;
  a.G = C.G;
  a.glog2 = C.glog2;
  a.ngroups = C.ngroups;
  a.npad = (int64_t)g->nparts * (int64_t)g->S;
  a.src = nullptr;
  a.D = C.D.as<uint32_t>();
  a.pend = C.pend.as<uint32_t>();
  a.dirty = C.dirty.as<uint32_t>();
  a.items = C.items.as<uint4>();
  a.hub_cap = (uint32_t)((uint64_t)C.ngroups * g->hub_chunks);
  a.hubs = g->nhubs ? g->hubs.as<uint32_t>() : nullptr;
  a.nhubs = g->nhubs;
  a.hub_chunk = kHubChunk;
  a.window = 0u;  // lanes of one group are of different ages: no shared window
  a.gbest = nullptr;
  a.ctrl = C.ctrl.as<Ctrl>();
  // a launch yields after max_rounds rounds (default 4,096) and the next one
  // resumes the same state, so no launch runs for long
  a.max_rounds = o.max_rounds ? o.max_rounds : 4096u;
  a.watchdog_ns = (uint64_t)(o.watchdog_ms ? o.watchdog_ms : 30000u) * 1000000ull;
  a.box = C.box_dev;
  a.res = C.res.as<uint32_t>();
  a.occ = C.occ.as<uint32_t>();
  a.seen = C.seen.as<uint32_t>();
  a.gact = C.gact.as<uint32_t>();
  a.init = C.need_init ? 1u : 0u;
  a.reach = C.qtype == Q_BFS ? C.reach.as<uint32_t>() : nullptr;
  a.lstart = C.qtype == Q_BFS ? C.lstart.as<uint32_t>() : nullptr;
  if (C.need_init) C.round0 = 0;
  a.round0 = C.round0;
  CUDA_TRY(launch_group(a, C.blocks, g->group_threads[C.gi], g->group_smem[C.gi], C.stream));
  CUDA_TRY(cudaMemcpyAsync(C.h_ctrl, C.ctrl.p, sizeof(Ctrl), cudaMemcpyDeviceToHost, C.stream));
  CUDA_TRY(cudaEventRecord(C.done_ev, C.stream));
  C.need_init = false;
  C.running = true;
  return FG_OK;
}

void finish_request(fg_server *s, uint64_t id, fg_status st, int64_t t) {
  Request &r = s->reqs[id];
  r.done = true;
  r.done_ns = t;
  r.status = st;
  s->finished.push_back(id);
}

// One progress step of a slot lane: completions posted in the mailbox, the end
// of the running launch, admission of waiting requests into free slots, and a
// new launch when a slot holds a request that no launch will see.
fg_status poll_slot_lane(fg_server *s, SlotLane &C) {
  fg_status first = FG_OK;
  bool ended = false;
  fg_status launch_st = FG_OK;
  if (C.running) {
    const cudaError_t q = cudaEventQuery(C.done_ev);
    if (q != cudaErrorNotReady) {
      C.running = false;
      ended = true;
      C.round0 += (uint32_t)C.h_ctrl->rounds;
      if (q != cudaSuccess) launch_st = fail(FG_ERR_CUDA, "slot lane: %s", cudaGetErrorString(q));
      else if (C.h_ctrl->status != 0)
        launch_st = fail((fg_status)C.h_ctrl->status, "slot lane: device reported status %d (site %u)",
                         C.h_ctrl->status, C.h_ctrl->site);
    }
  }
  const int64_t t = now_ns();
  for (int sl = 0; sl < C.nslots; ++sl) {
    if (C.slot_req[(size_t)sl] == 0 || C.slot_done[(size_t)sl]) continue;
    ServeSlot &b = C.box->slot[sl];
    if (__atomic_load_n(&b.done_seq, __ATOMIC_ACQUIRE) != C.slot_seq[(size_t)sl]) continue;
    const fg_status st = (fg_status)__atomic_load_n(&b.status, __ATOMIC_RELAXED);
    C.slot_done[(size_t)sl] = 1;
    finish_request(s, C.slot_req[(size_t)sl], st, t);
    if (st != FG_OK && first == FG_OK) first = fail(st, "slot lane: request rejected by the device");
  }
  if (ended && launch_st != FG_OK) {
    // the launch failed: its unfinished requests complete with its status, and
    // the next launch starts from a cleared state and mailbox
    for (int sl = 0; sl < C.nslots; ++sl) {
      if (C.slot_req[(size_t)sl] == 0 || C.slot_done[(size_t)sl]) continue;
      C.slot_done[(size_t)sl] = 1;
      finish_request(s, C.slot_req[(size_t)sl], launch_st, t);
    }
    std::memset(C.box->slot, 0, sizeof(ServeSlot) * (size_t)C.nslots);
    std::fill(C.slot_seq.begin(), C.slot_seq.end(), 0u);
    C.need_init = true;
    if (first == FG_OK) first = launch_st;
  }
  std::deque<uint64_t> &q = s->queue[C.kind];
  for (int sl = 0; sl < C.nslots && !q.empty(); ++sl) {
    if (C.slot_req[(size_t)sl] != 0) continue;
    const uint64_t id = q.front();
    q.pop_front();
    Request &r = s->reqs[id];
    r.slot = sl;
    r.row = sl;
    r.batch = C.nslots;
    r.launch_ns = t;
    ServeSlot &b = C.box->slot[sl];
    __atomic_store_n(&b.src, r.source, __ATOMIC_RELAXED);
    const uint32_t seq = C.slot_seq[(size_t)sl] + 1u;
    C.slot_seq[(size_t)sl] = seq;
    __atomic_store_n(&b.seq, seq, __ATOMIC_RELEASE);  // the source is visible before the sequence number
    C.slot_req[(size_t)sl] = id;
    C.slot_done[(size_t)sl] = 0;
  }
  if (!C.running) {
    // a slot holds a request not yet completed: either it waits in the mailbox
    // or the last launch yielded with it in flight
    bool waiting = false;
    for (int sl = 0; sl < C.nslots && !waiting; ++sl) waiting = C.slot_req[(size_t)sl] != 0 && !C.slot_done[(size_t)sl];
    if (waiting) {
      const fg_status st = launch_slot_lane(s, C);
      if (st != FG_OK) {
        for (int sl = 0; sl < C.nslots; ++sl) {
          if (C.slot_req[(size_t)sl] == 0 || C.slot_done[(size_t)sl]) continue;
          C.slot_done[(size_t)sl] = 1;
          finish_request(s, C.slot_req[(size_t)sl], st, t);
        }
        std::memset(C.box->slot, 0, sizeof(ServeSlot) * (size_t)C.nslots);
        std::fill(C.slot_seq.begin(), C.slot_seq.end(), 0u);
        C.need_init = true;
        if (first == FG_OK) first = st;
      }
    }
  }
  return first;
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
  if (o.continuous != 0 && o.continuous != 1) return fail(FG_ERR_INVALID_ARG, "continuous must be 0 or 1");
  int slot_G = 32;
  if (o.continuous) {
    const int32_t gs = o.opts[FG_QUERY_SSSP].group;
    slot_G = (gs == 8 || gs == 16 || gs == 32) ? gs : 32;
    if (o.slots < slot_G || o.slots % slot_G != 0)
      return fail(FG_ERR_INVALID_ARG, "slots must be a positive multiple of the group size %d", slot_G);
  }
  CUDA_TRY(cudaSetDevice(g->device));
  // admission by HBM budget: every lane must be able to hold a full batch of
  // the most expensive kind; under slot-level batching the two slot lanes
  // take half of it and the batch lanes (PPR) the rest
  int64_t budget = o.hbm_budget;
  if (budget == 0) {
    size_t fr = 0, tot = 0;
    CUDA_TRY(cudaMemGetInfo(&fr, &tot));
    budget = (int64_t)(0.6 * (double)fr);
  }
  if (o.continuous) {
    const double per_slot = per_slot_bytes(g, slot_G);
    const int64_t fit_slots = (int64_t)(0.5 * (double)budget / (2.0 * per_slot)) / slot_G * slot_G;
    if (fit_slots < slot_G)
      return fail(FG_ERR_OOM, "HBM budget %lld B holds no group of slots", (long long)budget);
    o.slots = (int32_t)std::min<int64_t>(o.slots, fit_slots);
    budget -= (int64_t)(2.0 * per_slot * (double)o.slots);
  }
  const double per_q = o.continuous ? per_request_bytes(g, FG_QUERY_PPR)
                                    : std::max(per_request_bytes(g, FG_QUERY_PPR), per_request_bytes(g, FG_QUERY_SSSP));
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
  if (st == FG_OK && o.continuous) {
    // the two slot lanes and the batch lanes share the resident grid
    const int div = o.full_grid ? 1 : o.lanes + 2;
    st = create_slot_lane(s, s->slot_lanes[0], FG_QUERY_SSSP, o.slots, slot_G, div);
    if (st == FG_OK) st = create_slot_lane(s, s->slot_lanes[1], FG_QUERY_BFS, o.slots, slot_G, div);
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
  for (SlotLane &C : s->slot_lanes) {
    if (C.box) __atomic_store_n(&C.box->stop, 1u, __ATOMIC_RELEASE);  // a running launch leaves at its next round
    if (C.stream) cudaStreamSynchronize(C.stream);
    C.release_all();
  }
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
  // 2. slot lanes: completions, admissions into free slots, relaunch
  if (s->o.continuous)
    for (SlotLane &C : s->slot_lanes) {
      const fg_status st = poll_slot_lane(s, C);
      if (st != FG_OK && first == FG_OK) first = st;
    }
  // 3. free lanes take the waiting requests of the kind that has waited longest
  for (Lane &L : s->lanes) {
    if (L.running || L.live > 0) continue;
    int kind = -1;
    int64_t oldest = 0;
    for (int k = 0; k < 3; ++k) {
      if (s->o.continuous && k != FG_QUERY_PPR) continue;  // SSSP and BFS go to the slot lanes
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
  if (r.done && r.slot >= 0 && r.status == FG_OK) {
    const SlotLane &C = s->slot_lanes[r.kind == FG_QUERY_BFS ? 1 : 0];
    info->result = C.res.as<uint32_t>() + (size_t)r.slot * (size_t)s->g->n;
  } else if (r.done && r.lane >= 0) {
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
  const int lane = it->second.lane, slot = it->second.slot;
  if (slot >= 0) s->slot_lanes[it->second.kind == FG_QUERY_BFS ? 1 : 0].slot_req[(size_t)slot] = 0;
  s->reqs.erase(it);
  if (lane >= 0) s->lanes[(size_t)lane].live -= 1;
  return FG_OK;
}
