// Autotuner: times candidate fg_opts for one query kind on a sample batch and
// keeps the fastest. For SSSP and BFS it first picks the query group (one query
// per warp, or the group engine with 16 or 32 lanes), which decides more than
// any other knob: on graphs whose partitions are cut by nearly every arc the
// group engine wins, on road-like graphs one query per warp does. Then:
//   - one query per warp: the window of FG_SCHED_PRIORITY, whose best value
//     differs by orders of magnitude between graph families (a few weight units
//     on a low-diameter R-MAT graph, ten mean weights on a road-like grid), so
//     candidates are scaled by the graph's mean arc weight (SSSP) or counted in
//     levels (BFS) and tried from the widest down until one takes more than
//     twice the best time; then yield heuristic 2 (delta = half and a quarter
//     of the window); on graphs with out-degree <= 8 the lane-per-vertex
//     expansion;
//   - group engine (SSSP): a per-group window of 16 and 4 mean weights;
//   - both: half the batch per launch (query_batch), which keeps a smaller
//     working set.
#include <cstring>
#include <vector>

#include "fg_host.h"

using namespace fg;

namespace {

fg_status time_batch(fg_graph *g, int kind, const int32_t *src, int32_t nq, void *dst, float *p, void *stream,
                     const fg_opts &o, float alpha, float eps, cudaEvent_t a, cudaEvent_t b, float *ms) {
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  CUDA_TRY(cudaEventRecord(a, s));
  fg_status st;
  if (kind == FG_QUERY_PPR)
    st = fg_ppr_batch(g, src, nq, alpha, eps, p, nullptr, nullptr, stream, &o);
  else if (kind == FG_QUERY_BFS)
    st = fg_bfs_batch(g, src, nq, static_cast<uint32_t *>(dst), stream, &o);
  else
    st = fg_sssp_batch(g, src, nq, static_cast<uint32_t *>(dst), stream, &o);
  if (st != FG_OK) return st;
  CUDA_TRY(cudaEventRecord(b, s));
  st = fg_sync(stream);
  if (st != FG_OK) return st;
  CUDA_TRY(cudaEventElapsedTime(ms, a, b));
  return FG_OK;
}

}  // namespace

extern "C" fg_status fg_tune_opts(fg_graph *g, int32_t kind, const int32_t *src, int32_t nq, void *stream,
                                  fg_opts *best, fg_tune_report *report) {
  return fg_tune_opts_ex(g, kind, src, nq, 0.15f, 1e-6f, stream, best, report);
}

extern "C" fg_status fg_tune_opts_ex(fg_graph *g, int32_t kind, const int32_t *src, int32_t nq, float alpha,
                                     float eps, void *stream, fg_opts *best, fg_tune_report *report) {
  if (!g || !src || !best) return fail(FG_ERR_INVALID_ARG, "NULL argument");
  if (nq <= 0) return fail(FG_ERR_INVALID_ARG, "nq must be > 0");
  if (kind < FG_QUERY_SSSP || kind > FG_QUERY_PPR) return fail(FG_ERR_INVALID_ARG, "unknown query kind %d", kind);
  if (kind == FG_QUERY_PPR && !(alpha > 0.f && alpha < 1.f)) return fail(FG_ERR_INVALID_ARG, "alpha must be in (0, 1)");
  if (kind == FG_QUERY_PPR && !(eps > 0.f)) return fail(FG_ERR_INVALID_ARG, "eps must be > 0");
  int bucket = 0;
  while ((1 << bucket) < nq && bucket < 30) ++bucket;
  // PPR choices are cached per (alpha, eps) as well
  uint32_t ab = 0, eb = 0;
  if (kind == FG_QUERY_PPR) {
    std::memcpy(&ab, &alpha, 4);
    std::memcpy(&eb, &eps, 4);
  }
  const TuneKey key{kind, bucket, ab, eb};
  {
    std::lock_guard<std::mutex> lk(g->mu);
    auto it = g->tuned.find(key);
    if (it != g->tuned.end()) {
      *best = it->second.first;
      if (report) {
        *report = it->second.second;
        report->candidates = 0;  // served from the cache
      }
      return FG_OK;
    }
  }
  CUDA_TRY(cudaSetDevice(g->device));
  DevBuf out;
  CUDA_TRY(out.reserve(4 * (size_t)nq * (size_t)g->n));
  cudaEvent_t ea = nullptr, eb_ = nullptr;
  CUDA_TRY(cudaEventCreate(&ea));
  CUDA_TRY(cudaEventCreate(&eb_));
  struct Guard {
    cudaEvent_t a, b;
    DevBuf *o;
    ~Guard() {
      cudaEventDestroy(a);
      cudaEventDestroy(b);
      o->release();
    }
  } guard{ea, eb_, &out};

  fg_opts base;
  fg_default_opts(&base);
  float ms = 0.f;
  int tried = 0;
  // one untimed run loads the kernels and sizes the workspace
  fg_status st = time_batch(g, kind, src, nq, out.p, out.as<float>(), stream, base, alpha, eps, ea, eb_, &ms);
  if (st != FG_OK) return st;
  st = time_batch(g, kind, src, nq, out.p, out.as<float>(), stream, base, alpha, eps, ea, eb_, &ms);
  if (st != FG_OK) return st;
  ++tried;
  fg_opts pick = base;
  float pick_ms = ms;
  const float base_ms = ms;

  auto try_opts = [&](const fg_opts &o) -> fg_status {
    float t = 0.f;
    fg_status s2 = time_batch(g, kind, src, nq, out.p, nullptr, stream, o, alpha, eps, ea, eb_, &t);
    if (s2 != FG_OK) return s2;
    ++tried;
    if (t < pick_ms) {
      pick = o;
      pick_ms = t;
    }
    ms = t;
    return FG_OK;
  };
  // the query group (what the default resolves to is measured already)
  const int auto_group = auto_group_size(g, kind == FG_QUERY_BFS ? Q_BFS : Q_SSSP, nq, false);
  if (kind != FG_QUERY_PPR) {
    for (int G : {1, 16, 32, 64}) {
      if (G == auto_group || (G > 1 && !group_fits(g->S, G))) continue;
      fg_opts o = base;
      o.group = G;
      if ((st = try_opts(o)) != FG_OK) return st;
    }
    if (pick.group == 0) pick.group = auto_group;
  }
  if (kind != FG_QUERY_PPR && pick.group > 1) {
    // group engine: a per-group window (Delta-stepping across rounds) for SSSP
    if (kind == FG_QUERY_SSSP && g->weighted && pick.group != 64) {  // groups of 64 run FIFO rounds only
      const fg_opts chosen = pick;
      for (double f : {16.0, 4.0}) {
        fg_opts o = chosen;
        o.sched = FG_SCHED_PRIORITY;
        o.sched_window = (uint32_t)(f * g->mean_weight + 0.5);
        if ((st = try_opts(o)) != FG_OK) return st;
      }
    }
  }
  if (kind != FG_QUERY_PPR) {  // PPR buffers are scheduled first-in first-out
    // one query per warp with per-query windows, from wide to narrow, against
    // whatever has won so far: a FIFO group engine can beat one query per
    // warp in FIFO rounds on a road-like graph and still lose to its windows
    std::vector<double> windows;
    if (kind == FG_QUERY_BFS || !g->weighted) {
      const double lv[] = {64, 48, 32, 24, 16, 12, 8, 4, 2};
      windows.assign(lv, lv + sizeof(lv) / sizeof(lv[0]));
    } else {
      const double f[] = {16, 10, 6, 4, 2, 1, 0.5, 0.25, 0.125, 1.0 / 16, 1.0 / 32, 1.0 / 64, 1.0 / 128};
      for (double x : f) windows.push_back(x * g->mean_weight);
    }
    uint32_t last = 0;
    for (double wd : windows) {
      const uint32_t w = (uint32_t)(wd < 1.0 ? 1.0 : wd + 0.5);
      if (w == last) continue;
      last = w;
      fg_opts o = base;
      o.group = 1;
      o.sched = FG_SCHED_PRIORITY;
      o.sched_window = w;
      st = time_batch(g, kind, src, nq, out.p, nullptr, stream, o, alpha, eps, ea, eb_, &ms);
      if (st != FG_OK) return st;
      ++tried;
      if (ms < pick_ms) {
        pick = o;
        pick_ms = ms;
      } else if (ms > 2.f * pick_ms) {
        break;  // narrower windows only add rounds from here on
      }
    }
    // yield heuristic 2 on top of the chosen window: values beyond (first value
    // + delta) wait for a later visit
    if (pick.group == 1 && pick.sched == FG_SCHED_PRIORITY) {
      const uint32_t w = pick.sched_window;
      for (uint32_t dl : {w / 2u, w / 4u}) {
        if (dl == 0u) continue;
        fg_opts o = pick;
        o.delta = dl;
        st = time_batch(g, kind, src, nq, out.p, nullptr, stream, o, alpha, eps, ea, eb_, &ms);
        if (st != FG_OK) return st;
        ++tried;
        if (ms < pick_ms) {
          pick = o;
          pick_ms = ms;
        }
      }
    }
    if (pick.group == 1 && g->max_degree <= 8) {
      fg_opts o = pick;
      o.threads_per_vertex = 1;
      st = time_batch(g, kind, src, nq, out.p, nullptr, stream, o, alpha, eps, ea, eb_, &ms);
      if (st != FG_OK) return st;
      ++tried;
      if (ms < pick_ms) {
        pick = o;
        pick_ms = ms;
      }
    }
  }
  // half the batch per launch
  if (nq >= 64) {
    fg_opts o = pick;
    o.query_batch = (nq / 2 + 31) / 32 * 32;
    if ((st = try_opts(o)) != FG_OK) return st;
  }
  *best = pick;
  fg_tune_report r;
  r.candidates = tried;
  r.best_ms = pick_ms;
  r.default_ms = base_ms;
  if (report) *report = r;
  {
    std::lock_guard<std::mutex> lk(g->mu);
    g->tuned[key] = std::make_pair(pick, r);
  }
  return FG_OK;
}
