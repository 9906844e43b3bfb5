// Host runtime behind the C ABI of include/fg.h: argument checks, graph
// partitioning and upload, per-graph device workspace, batch launches and the
// status / statistics path of fg_sync.
#include <algorithm>
#include <cstdarg>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "fg_host.h"

namespace fg {
bool partition_plan_impl(int64_t n, const int64_t *row_ptr, const int32_t *col, int method, int S, int32_t *perm);
int64_t cut_arcs_impl(int64_t n, const int64_t *row_ptr, const int32_t *col, const int32_t *perm, int slog2);
}  // namespace fg

using namespace fg;

namespace {
thread_local std::string t_err;
}  // namespace

namespace fg {
fg_status fail(fg_status s, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  t_err = buf;
  return s;
}
}  // namespace fg

namespace {

// A batch whose status fg_sync has not read yet.
struct Pending {
  cudaStream_t stream;
  fg_graph *graph;
  Workspace *ws;  // workspace the batch ran on (its pending bitmaps need a reset after an abort)
  Ctrl *host;     // pinned copy of the device control block
  unsigned launches;
  unsigned group;  // queries per group of the batch's launches
};

std::mutex g_pending_mu;
std::vector<Pending> g_pending;
std::vector<Ctrl *> g_slot_pool;  // pinned status slots ready for reuse (guarded by g_pending_mu)

Ctrl *take_slot() {
  {
    std::lock_guard<std::mutex> lp(g_pending_mu);
    if (!g_slot_pool.empty()) {
      Ctrl *h = g_slot_pool.back();
      g_slot_pool.pop_back();
      return h;
    }
  }
  Ctrl *h = nullptr;
  if (cudaMallocHost(&h, sizeof(Ctrl)) != cudaSuccess) return nullptr;
  return h;
}

}  // namespace

extern "C" void fg_default_opts(fg_opts *o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->struct_size = sizeof(fg_opts);
  o->mode = FG_MODE_BUFFERED;
  o->sched = FG_SCHED_FIFO;
}

extern "C" void fg_default_graph_opts(fg_graph_opts *o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->struct_size = sizeof(fg_graph_opts);
  o->partition_method = FG_PART_AUTO;
}

extern "C" const char *fg_last_error(void) { return t_err.c_str(); }

static int ilog2(int64_t x) {
  int l = 0;
  while ((int64_t(1) << (l + 1)) <= x) ++l;
  return l;
}

// Partition size from the measured on-chip budget: each resident warp keeps
// one query's slice (S values + five S-bit bitmaps) in shared memory, and an
// SM should hold at least 32 such warps.
static int default_partition_vertices() {
  int dev = 0, smem_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 1024;
  if (cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess)
    return 1024;
  const double per_vertex = 4.0 + 5.0 / 8.0;
  int64_t s = (int64_t)(smem_sm / (32 * per_vertex));
  int S = 1 << ilog2(std::max<int64_t>(32, s));
  return std::min(4096, std::max(32, S));
}

extern "C" fg_status fg_partition_plan(int64_t n, const int64_t *row_ptr, const int32_t *col, int32_t method,
                                       int32_t partition_vertices, int32_t *perm) {
  if (n < 1 || n >= (int64_t(1) << 31) || !perm || partition_vertices < 1)
    return fail(FG_ERR_INVALID_ARG, "fg_partition_plan: bad arguments");
  if (method != FG_PART_RANGE && method != FG_PART_GROW && method != FG_PART_DEGREE)
    return fail(FG_ERR_INVALID_ARG, "fg_partition_plan: method must be FG_PART_RANGE, FG_PART_GROW or FG_PART_DEGREE");
  if ((method == FG_PART_GROW && !col) || (method != FG_PART_RANGE && !row_ptr))
    return fail(FG_ERR_INVALID_ARG, "fg_partition_plan: GROW and DEGREE need the CSR");
  if (!partition_plan_impl(n, row_ptr, col, method, partition_vertices, perm))
    return fail(FG_ERR_INVALID_ARG, "fg_partition_plan failed");
  return FG_OK;
}

static fg_status validate_csr(int64_t n, int64_t m, const int64_t *row_ptr, const int32_t *col, const int32_t *w) {
  if (n < 1 || n >= (int64_t(1) << 31)) return fail(FG_ERR_INVALID_ARG, "n must be in [1, 2^31)");
  if (m < 0) return fail(FG_ERR_INVALID_ARG, "m must be >= 0");
  if (m >= (int64_t(1) << 32)) return fail(FG_ERR_UNSUPPORTED, "m must be < 2^32");
  if (!row_ptr) return fail(FG_ERR_INVALID_ARG, "row_ptr is NULL");
  if (m > 0 && !col) return fail(FG_ERR_INVALID_ARG, "col is NULL");
  if (row_ptr[0] != 0 || row_ptr[n] != m) return fail(FG_ERR_INVALID_ARG, "row_ptr[0] must be 0 and row_ptr[n] = m");
  for (int64_t v = 0; v < n; ++v)
    if (row_ptr[v + 1] < row_ptr[v]) return fail(FG_ERR_INVALID_ARG, "row_ptr decreases at %lld", (long long)v);
  for (int64_t e = 0; e < m; ++e)
    if (col[e] < 0 || col[e] >= n) return fail(FG_ERR_INVALID_ARG, "col[%lld] = %d out of range", (long long)e, col[e]);
  if (w)
    for (int64_t e = 0; e < m; ++e)
      if (w[e] < 0) return fail(FG_ERR_INVALID_ARG, "negative weight w[%lld] = %d", (long long)e, w[e]);
  return FG_OK;
}

extern "C" fg_status fg_graph_create(int64_t n, int64_t m, const int64_t *row_ptr, const int32_t *col,
                                     const int32_t *w, uint32_t flags, fg_graph **out) {
  return fg_graph_create_ex(n, m, row_ptr, col, w, flags, nullptr, out);
}

extern "C" fg_status fg_graph_create_ex(int64_t n, int64_t m, const int64_t *row_ptr, const int32_t *col,
                                        const int32_t *w, uint32_t flags, const fg_graph_opts *gopts_in,
                                        fg_graph **out) {
  if (!out) return fail(FG_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  fg_graph_opts go;
  fg_default_graph_opts(&go);
  if (gopts_in) {
    if (gopts_in->struct_size < sizeof(uint32_t) + 2 * sizeof(int32_t))
      return fail(FG_ERR_INVALID_ARG, "fg_graph_opts.struct_size too small");
    go.partition_method = gopts_in->partition_method;
    go.partition_vertices = gopts_in->partition_vertices;
  }
  if (go.partition_method < FG_PART_AUTO || go.partition_method > FG_PART_DEGREE)
    return fail(FG_ERR_INVALID_ARG, "unknown partition method %d", go.partition_method);
  if (go.partition_vertices != 0 &&
      (go.partition_vertices < 32 || go.partition_vertices > 4096 ||
       (go.partition_vertices & (go.partition_vertices - 1)) != 0))
    return fail(FG_ERR_INVALID_ARG, "partition_vertices must be 0 or a power of two in [32, 4096]");
  if (n < 1 || n >= (int64_t(1) << 31)) return fail(FG_ERR_INVALID_ARG, "n must be in [1, 2^31)");
  if (m < 0) return fail(FG_ERR_INVALID_ARG, "m must be >= 0");
  if (m >= (int64_t(1) << 32)) return fail(FG_ERR_UNSUPPORTED, "m must be < 2^32");

  // host copies of the CSR
  std::vector<int64_t> h_rp;
  std::vector<int32_t> h_col, h_w;
  const int64_t *rp = row_ptr;
  const int32_t *cl = col, *wt = w;
  if (flags & FG_DEVICE_PTRS) {
    if (!row_ptr || (m > 0 && !col)) return fail(FG_ERR_INVALID_ARG, "NULL device pointer");
    h_rp.resize((size_t)n + 1);
    h_col.resize((size_t)std::max<int64_t>(m, 1));
    CUDA_TRY(cudaMemcpy(h_rp.data(), row_ptr, sizeof(int64_t) * (size_t)(n + 1), cudaMemcpyDeviceToHost));
    if (m > 0) CUDA_TRY(cudaMemcpy(h_col.data(), col, sizeof(int32_t) * (size_t)m, cudaMemcpyDeviceToHost));
    if (w) {
      h_w.resize((size_t)std::max<int64_t>(m, 1));
      if (m > 0) CUDA_TRY(cudaMemcpy(h_w.data(), w, sizeof(int32_t) * (size_t)m, cudaMemcpyDeviceToHost));
    }
    rp = h_rp.data();
    cl = h_col.data();
    wt = w ? h_w.data() : nullptr;
  }
  fg_status st = validate_csr(n, m, rp, cl, wt);
  if (st != FG_OK) return st;

  int dev = 0;
  CUDA_TRY(cudaGetDevice(&dev));
  int S = go.partition_vertices ? go.partition_vertices : default_partition_vertices();
  while (S > 32 && (int64_t)S / 2 >= n) S /= 2;  // no partition larger than needed
  const int slog2 = ilog2(S);

  // partition: AUTO keeps the id order unless breadth-first growth cuts far fewer arcs
  std::vector<int32_t> perm((size_t)n);
  int method = go.partition_method;
  int64_t cut = 0;
  if (method == FG_PART_AUTO) {
    partition_plan_impl(n, rp, cl, FG_PART_RANGE, S, perm.data());
    const int64_t cut_range = cut_arcs_impl(n, rp, cl, perm.data(), slog2);
    method = FG_PART_RANGE;
    cut = cut_range;
    if (m > 0 && (double)cut_range / (double)m > 0.25) {
      std::vector<int32_t> perm2((size_t)n);
      partition_plan_impl(n, rp, cl, FG_PART_GROW, S, perm2.data());
      const int64_t cut_grow = cut_arcs_impl(n, rp, cl, perm2.data(), slog2);
      if (cut_grow < cut_range * 7 / 10) {
        perm.swap(perm2);
        method = FG_PART_GROW;
        cut = cut_grow;
      }
    }
  } else {
    partition_plan_impl(n, rp, cl, method, S, perm.data());
    cut = cut_arcs_impl(n, rp, cl, perm.data(), slog2);
  }
  const bool identity = (method == FG_PART_RANGE);

  // internal (partition-major) CSR with 32-bit offsets
  std::vector<uint32_t> i_rp((size_t)n + 1), i_adj((size_t)std::max<int64_t>(m, 1)), i_wt;
  std::vector<int32_t> intl;
  if (wt) i_wt.resize((size_t)std::max<int64_t>(m, 1));
  if (identity) {
    for (int64_t v = 0; v <= n; ++v) i_rp[(size_t)v] = (uint32_t)rp[v];
    for (int64_t e = 0; e < m; ++e) i_adj[(size_t)e] = (uint32_t)cl[e];
    if (wt)
      for (int64_t e = 0; e < m; ++e) i_wt[(size_t)e] = (uint32_t)wt[e];
  } else {
    intl.resize((size_t)n);
    for (int64_t i = 0; i < n; ++i) intl[(size_t)perm[(size_t)i]] = (int32_t)i;
    uint64_t k = 0;
    for (int64_t i = 0; i < n; ++i) {
      i_rp[(size_t)i] = (uint32_t)k;
      const int32_t v = perm[(size_t)i];
      for (int64_t e = rp[v]; e < rp[v + 1]; ++e) {
        i_adj[k] = (uint32_t)intl[(size_t)cl[e]];
        if (wt) i_wt[k] = (uint32_t)wt[e];
        ++k;
      }
    }
    i_rp[(size_t)n] = (uint32_t)k;
  }

  fg_graph *g = new (std::nothrow) fg_graph();
  if (!g) return fail(FG_ERR_OOM, "host allocation failed");
  g->n = n;
  g->m = m;
  g->method = method;
  g->S = S;
  g->slog2 = slog2;
  g->nparts = (int)((n + S - 1) / S);
  g->cut = cut;
  g->weighted = wt != nullptr;
  g->device = dev;
  auto cleanup = [&](fg_status s) {
    g->rp.release(); g->adj.release(); g->wt.release(); g->orig.release(); g->intl.release();
    g->hubs.release();
    delete g;
    return s;
  };
#define CUDA_TRY_G(expr)                                                                      \
  do {                                                                                        \
    cudaError_t e_ = (expr);                                                                  \
    if (e_ != cudaSuccess)                                                                    \
      return cleanup(fail(e_ == cudaErrorMemoryAllocation ? FG_ERR_OOM : FG_ERR_CUDA, "%s: %s", #expr, \
                          cudaGetErrorString(e_)));                                           \
  } while (0)
  // a partition's row offsets are read as rp[base, base + S] (S + 1 entries), so
  // rp is padded to whole partitions; adj / wt get a small tail pad
  const size_t rp_elems = (size_t)g->nparts * (size_t)S + 64, arc_elems = (size_t)m + 64;
  CUDA_TRY_G(g->rp.reserve(sizeof(uint32_t) * rp_elems));
  CUDA_TRY_G(g->adj.reserve(sizeof(uint32_t) * arc_elems));
  CUDA_TRY_G(cudaMemset(g->rp.p, 0, sizeof(uint32_t) * rp_elems));
  CUDA_TRY_G(cudaMemset(g->adj.p, 0, sizeof(uint32_t) * arc_elems));
  CUDA_TRY_G(cudaMemcpy(g->rp.p, i_rp.data(), sizeof(uint32_t) * (size_t)(n + 1), cudaMemcpyHostToDevice));
  if (m > 0) CUDA_TRY_G(cudaMemcpy(g->adj.p, i_adj.data(), sizeof(uint32_t) * (size_t)m, cudaMemcpyHostToDevice));
  g->graph_bytes = sizeof(uint32_t) * (size_t)(n + 1 + m);
  if (wt) {
    CUDA_TRY_G(g->wt.reserve(sizeof(uint32_t) * arc_elems));
    CUDA_TRY_G(cudaMemset(g->wt.p, 0, sizeof(uint32_t) * arc_elems));
    if (m > 0) CUDA_TRY_G(cudaMemcpy(g->wt.p, i_wt.data(), sizeof(uint32_t) * (size_t)m, cudaMemcpyHostToDevice));
    g->graph_bytes += sizeof(uint32_t) * (size_t)m;
    double sum = 0.0;
    for (int64_t e = 0; e < m; ++e) {
      sum += (double)i_wt[(size_t)e];
      if (i_wt[(size_t)e] == 0u) g->has_zero_weight = true;
      g->max_weight = std::max(g->max_weight, i_wt[(size_t)e]);
    }
    if (m > 0) g->mean_weight = sum / (double)m;
  }
  std::vector<uint32_t> hubs;
  for (int64_t v = 0; v < n; ++v) {
    const uint32_t deg = i_rp[(size_t)v + 1] - i_rp[(size_t)v];
    g->max_degree = std::max(g->max_degree, deg);
    if (deg > kHubMin) {
      hubs.push_back((uint32_t)v);
      g->hub_chunks += (deg + kHubChunk - 1) / kHubChunk;
    }
  }
  g->nhubs = (int32_t)hubs.size();
  if (!hubs.empty()) {
    CUDA_TRY_G(g->hubs.reserve(sizeof(uint32_t) * hubs.size()));
    CUDA_TRY_G(cudaMemcpy(g->hubs.p, hubs.data(), sizeof(uint32_t) * hubs.size(), cudaMemcpyHostToDevice));
  }
  if (!identity) {
    CUDA_TRY_G(g->orig.reserve(sizeof(int32_t) * (size_t)n));
    CUDA_TRY_G(g->intl.reserve(sizeof(int32_t) * (size_t)n));
    CUDA_TRY_G(cudaMemcpy(g->orig.p, perm.data(), sizeof(int32_t) * (size_t)n, cudaMemcpyHostToDevice));
    CUDA_TRY_G(cudaMemcpy(g->intl.p, intl.data(), sizeof(int32_t) * (size_t)n, cudaMemcpyHostToDevice));
    g->graph_bytes += 2 * sizeof(int32_t) * (size_t)n;
  }
  CUDA_TRY_G(cudaEventCreateWithFlags(&g->last_done, cudaEventDisableTiming));
#undef CUDA_TRY_G
  DevGraph &d = g->dg;
  d.n = (int32_t)n;
  d.slog2 = slog2;
  d.S = S;
  d.nparts = g->nparts;
  d.m = (uint64_t)m;
  d.max_deg = g->max_degree;
  d.max_w = wt ? g->max_weight : 1u;
  d.rp = g->rp.as<uint32_t>();
  d.adj = g->adj.as<uint32_t>();
  d.wt = wt ? g->wt.as<uint32_t>() : nullptr;
  d.orig = identity ? nullptr : g->orig.as<int32_t>();
  d.intl = identity ? nullptr : g->intl.as<int32_t>();
  // the no-allocation entry point's scratch is placed on the device now, while
  // the caller's memory is still free (lazy module loading would otherwise
  // place it at that entry point's first call)
  noalloc_prepare(dev);
  *out = g;
  return FG_OK;
}

extern "C" fg_status fg_graph_destroy(fg_graph *g) {
  if (!g) return FG_OK;
  {
    std::lock_guard<std::mutex> lk(g->mu);
    cudaSetDevice(g->device);
    if (g->has_last) cudaEventSynchronize(g->last_done);
    {
      std::lock_guard<std::mutex> lp(g_pending_mu);
      for (auto &p : g_pending)
        if (p.graph == g) {
          p.graph = nullptr;
          p.ws = nullptr;
        }
    }
    g->ws.release_all();
    g->rp.release(); g->adj.release(); g->wt.release(); g->orig.release(); g->intl.release();
    g->deg.release();
    g->hubs.release();
    g->bc.release_all();
    g->dfs.release_all();
    if (g->last_done) cudaEventDestroy(g->last_done);
  }
  delete g;
  return FG_OK;
}

extern "C" fg_status fg_graph_info(const fg_graph *g, fg_graph_info_t *info) {
  if (!g || !info) return fail(FG_ERR_INVALID_ARG, "NULL argument");
  info->n = g->n;
  info->m = g->m;
  info->partition_vertices = g->S;
  info->num_partitions = g->nparts;
  info->partition_method = g->method;
  info->weighted = g->weighted ? 1 : 0;
  info->cut_arcs = g->cut;
  info->device_bytes = (int64_t)g->graph_bytes;
  return FG_OK;
}

extern "C" fg_status fg_stats(const fg_graph *g, fg_stats_t *out) {
  if (!g || !out) return fail(FG_ERR_INVALID_ARG, "NULL argument");
  *out = g->last_stats;
  return FG_OK;
}

static void merge_opts(const fg_opts *in, fg_opts *o) {
  fg_default_opts(o);
  if (!in) return;
  size_t sz = std::min<size_t>(in->struct_size, sizeof(fg_opts));
  if (sz > sizeof(uint32_t)) std::memcpy(reinterpret_cast<char *>(o) + sizeof(uint32_t),
                                         reinterpret_cast<const char *>(in) + sizeof(uint32_t), sz - sizeof(uint32_t));
  o->struct_size = sizeof(fg_opts);
}

namespace {

// workspace for a buffered launch of nb queries
fg_status ensure_engine_ws(fg_graph *g, Workspace &ws, int qtype, int64_t nb, uint64_t e_cap, bool need_r,
                           int blocks) {
  const bool relabelled = g->dg.orig != nullptr;
  const uint64_t K = (uint64_t)g->nparts * (uint64_t)nb;
  const uint64_t nw = (uint64_t)(g->S / 32);
  CUDA_TRY(ws.cnt.reserve(4 * K));
  CUDA_TRY(ws.prio.reserve(4 * K));
  CUDA_TRY(ws.dirty.reserve(4 * K));
  CUDA_TRY(ws.cur.reserve(4 * K));
  CUDA_TRY(ws.items.reserve(16 * K));
  CUDA_TRY(ws.iprio.reserve(4 * K));
  const size_t pend_bytes = 4 * K * nw;
  if (ws.pend.bytes < pend_bytes) {
    CUDA_TRY(ws.pend.reserve(pend_bytes));
    ws.pend_clean = false;
  }
  CUDA_TRY(ws.qbest.reserve(8 * (size_t)nb));
  CUDA_TRY(ws.blocksum.reserve(16 * (size_t)blocks));
  CUDA_TRY(ws.e_key.reserve(4 * e_cap));
  CUDA_TRY(ws.e_op.reserve(8 * e_cap));
  CUDA_TRY(ws.b_op.reserve(8 * e_cap));
  CUDA_TRY(ws.ctrl.reserve(sizeof(Ctrl)));
  const size_t rows = (size_t)nb * (size_t)g->n;
  if (qtype == Q_PPR) {
    // estimates, residuals (when not requested or relabelled) and Kahan terms
    CUDA_TRY(ws.scratch_c.reserve(4 * rows));
    if (need_r || relabelled) CUDA_TRY(ws.scratch_r.reserve(4 * rows));
    if (relabelled) CUDA_TRY(ws.scratch_p.reserve(4 * rows));
  } else if (relabelled) {
    CUDA_TRY(ws.state.reserve(4 * rows));  // distances in partition-major order
  }
  return FG_OK;
}

fg_status ensure_plain_ws(fg_graph *g, Workspace &ws, int qtype, int64_t nb, bool need_r) {
  const size_t n = (size_t)g->n;
  CUDA_TRY(ws.ctrl.reserve(sizeof(Ctrl)));
  CUDA_TRY(ws.pl_stamp.reserve(4 * n));
  CUDA_TRY(ws.pl_f0.reserve(4 * n));
  CUDA_TRY(ws.pl_f1.reserve(4 * n));
  CUDA_TRY(ws.pl_sizes.reserve(16));
  if (qtype == Q_PPR) {
    CUDA_TRY(ws.pl_rr.reserve(4 * n));
    CUDA_TRY(ws.pl_pp.reserve(4 * n));
    CUDA_TRY(ws.pl_cc.reserve(4 * n));
    CUDA_TRY(ws.scratch_c.reserve(4 * (size_t)nb * n));
    if (need_r) CUDA_TRY(ws.scratch_r.reserve(4 * (size_t)nb * n));
  } else {
    CUDA_TRY(ws.pl_dist.reserve(4 * n));
  }
  return FG_OK;
}

}  // namespace

namespace fg {

// One batch on workspace ws. shared_ws: ws is the graph's own workspace, so
// the batch waits for the graph's previous batch (stream order across
// streams). grid_div > 1 launches the engine on 1/grid_div of the resident
// grid, so that several batches (server lanes) run side by side.
fg_status run_batch_on(fg_graph *g, Workspace &ws, bool shared_ws, int grid_div, int qtype, const int32_t *src_in,
                       int32_t nq, uint32_t *dist_in, float alpha, float eps, float *p_in, float *r_in,
                       double *mass_in, void *stream_v, const fg_opts *opts_in) {
  if (!g) return fail(FG_ERR_INVALID_ARG, "graph is NULL");
  if (nq <= 0) return fail(FG_ERR_INVALID_ARG, "nq must be > 0");
  if (!src_in) return fail(FG_ERR_INVALID_ARG, "src is NULL");
  if ((qtype != Q_PPR && !dist_in) || (qtype == Q_PPR && !p_in)) return fail(FG_ERR_INVALID_ARG, "output is NULL");
  if ((reinterpret_cast<uintptr_t>(src_in) & 3u) || (reinterpret_cast<uintptr_t>(dist_in) & 3u) ||
      (reinterpret_cast<uintptr_t>(p_in) & 3u) || (reinterpret_cast<uintptr_t>(r_in) & 3u) ||
      (reinterpret_cast<uintptr_t>(mass_in) & 7u))
    return fail(FG_ERR_INVALID_ARG, "misaligned pointer");
  if (qtype == Q_PPR && !(alpha > 0.f && alpha < 1.f)) return fail(FG_ERR_INVALID_ARG, "alpha must be in (0, 1)");
  if (qtype == Q_PPR && !(eps > 0.f)) return fail(FG_ERR_INVALID_ARG, "eps must be > 0");
  fg_opts o;
  merge_opts(opts_in, &o);
  if (o.mode != FG_MODE_BUFFERED && o.mode != FG_MODE_PLAIN) return fail(FG_ERR_INVALID_ARG, "unknown mode");
  if (o.sched < FG_SCHED_FIFO || o.sched > FG_SCHED_RANDOM) return fail(FG_ERR_INVALID_ARG, "unknown sched");
  if (o.query_batch < 0) return fail(FG_ERR_INVALID_ARG, "query_batch must be >= 0");
  if (o.host_io < 0 || o.host_io > 2) return fail(FG_ERR_INVALID_ARG, "host_io must be 0, 1 or 2");
  if (o.threads_per_vertex != 0 && o.threads_per_vertex != 1 && o.threads_per_vertex != 32)
    return fail(FG_ERR_INVALID_ARG, "threads_per_vertex must be 0, 1 or 32");
  if (o.group != 0 && o.group != 1 && o.group != 8 && o.group != 16 && o.group != 32 && o.group != 64)
    return fail(FG_ERR_INVALID_ARG, "group must be 0, 1, 8, 16, 32 or 64");
  if (o.group_order != 0 && o.group_order != 1) return fail(FG_ERR_INVALID_ARG, "group_order must be 0 or 1");
  if (o.check_staging != 0 && o.check_staging != 1) return fail(FG_ERR_INVALID_ARG, "check_staging must be 0 or 1");
  if (qtype == Q_PPR) o.sched = FG_SCHED_FIFO;  // PPR buffers are scheduled first-in first-out
  const uint32_t max_rounds = o.max_rounds ? o.max_rounds : 1000000u;
  const uint64_t watchdog_ns = (uint64_t)(o.watchdog_ms ? o.watchdog_ms : 30000u) * 1000000ull;
  const int64_t n = g->n;

  std::lock_guard<std::mutex> lk(g->mu);
  CUDA_TRY(cudaSetDevice(g->device));
  cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_v);

  // host I/O: validate and stage the sources, stage outputs on the device
  const int32_t *src = src_in;
  uint32_t *dist = dist_in;
  float *pout = p_in, *rout = r_in;
  double *mass = mass_in;
  const bool host_io = o.host_io != 0;
  const size_t row_elems = (size_t)nq * (size_t)n;
  IoSlot *io = nullptr;
  if (host_io) {
    for (int32_t i = 0; i < nq; ++i)
      if (src_in[i] < 0 || src_in[i] >= n)
        return fail(FG_ERR_INVALID_ARG, "src[%d] = %d out of range", i, src_in[i]);
    // staging slots are used in turn; before a slot is refilled on this
    // stream, its previous copy to the host (on whatever stream) must be done
    io = &ws.io[ws.io_next];
    ws.io_next ^= 1;
    if (!io->done) CUDA_TRY(cudaEventCreateWithFlags(&io->done, cudaEventDisableTiming));
    const size_t mass_off = ((4 * (size_t)nq + 15) / 16) * 16;
    const bool grow = io->src.bytes < mass_off + 8 * (size_t)nq || io->out.bytes < 4 * row_elems ||
                      (qtype == Q_PPR && r_in && io->out2.bytes < 4 * row_elems);
    if (io->used) {
      if (grow) CUDA_TRY(cudaEventSynchronize(io->done));  // reallocation frees the old buffers
      else CUDA_TRY(cudaStreamWaitEvent(stream, io->done, 0));
    }
    CUDA_TRY(io->src.reserve(mass_off + 8 * (size_t)nq));
    CUDA_TRY(io->out.reserve(4 * row_elems));
    if (qtype == Q_PPR && r_in) CUDA_TRY(io->out2.reserve(4 * row_elems));
    CUDA_TRY(cudaMemcpyAsync(io->src.p, src_in, 4 * (size_t)nq, cudaMemcpyHostToDevice, stream));
    src = io->src.as<int32_t>();
    mass = mass_in ? reinterpret_cast<double *>(io->src.as<char>() + mass_off) : nullptr;
    if (qtype == Q_PPR) {
      pout = io->out.as<float>();
      rout = r_in ? io->out2.as<float>() : nullptr;
    } else {
      dist = io->out.as<uint32_t>();
    }
  }
  if (shared_ws && g->has_last) CUDA_TRY(cudaStreamWaitEvent(stream, g->last_done, 0));
  const bool need_r = (qtype == Q_PPR && rout == nullptr);
  // queries per launch: bounded by the workspace (keys, pending bitmaps, PPR scratch)
  int64_t nb = o.query_batch ? o.query_batch : nq;
  {
    const bool relabelled = g->dg.orig != nullptr;
    const double per_query = (double)g->nparts * 36.0 + (double)n / 8.0 +
                             (qtype == Q_PPR ? (relabelled ? 12.0 : (need_r ? 8.0 : 4.0)) * (double)n
                                             : (relabelled ? 4.0 : 0.0) * (double)n);
    // the device's free memory (plus what this workspace already holds, which a
    // regrow frees first), less a margin; the arena is sized separately below
    size_t free_b = 0, total_b = 0;
    CUDA_TRY(cudaMemGetInfo(&free_b, &total_b));
    const size_t held = ws.cnt.bytes + ws.prio.bytes + ws.dirty.bytes + ws.cur.bytes + ws.pend.bytes +
                        ws.items.bytes + ws.iprio.bytes + ws.scratch_r.bytes + ws.scratch_c.bytes +
                        ws.scratch_p.bytes + ws.state.bytes;
    const double budget = std::max(0.0, 0.8 * (double)(free_b + held) - 12e9);
    const int64_t cap_q = std::max<int64_t>(1, (int64_t)(budget / per_query));
    nb = std::min<int64_t>(nb, cap_q);
    const int64_t key_cap = (int64_t)((0xFFFFFFFEull) / (uint64_t)g->nparts);
    nb = std::min<int64_t>(nb, key_cap);
    nb = std::min<int64_t>(nb, nq);
  }
  int launches = 0;
  Ctrl *d_ctrl = nullptr;
  // query group: one lane per query (group engine) where most arcs leave their
  // partition, else one warp per query and visit; PPR is never grouped
  int Gq = 1;
  if (qtype != Q_PPR && o.mode == FG_MODE_BUFFERED)
    Gq = o.group == 0 ? auto_group_size(g, qtype, nq, o.sched == FG_SCHED_PRIORITY && o.sched_window != 0u)
                      : o.group;

  if (o.mode == FG_MODE_BUFFERED && Gq > 1) {
    int glog2 = 0;
    while ((1 << glog2) < Gq) ++glog2;
    const int64_t npad = (int64_t)g->nparts * (int64_t)g->S;
    // queries per launch from the device's free memory: per group the state
    // (G values per vertex), two pending masks per vertex, the dirty flags and
    // work items of its partitions and its hub chunks
    int64_t nbq = o.query_batch ? o.query_batch : nq;
    {
      size_t free_b = 0, total_b = 0;
      CUDA_TRY(cudaMemGetInfo(&free_b, &total_b));
      const size_t held = ws.g_D.bytes + ws.g_pend.bytes + ws.g_dirty.bytes + ws.g_items.bytes + ws.g_best.bytes +
                          ws.g_reach.bytes;
      const double avail = 0.9 * (double)(free_b + held) - 512.0 * 1024 * 1024;
      const double mask_b = Gq == 64 ? 8.0 : 4.0;
      const double per_group = (double)npad * 4.0 * (double)Gq + (qtype == Q_BFS ? 3.0 : 2.0) * mask_b * (double)npad +
                               24.0 * (double)g->nparts + 20.0 * (double)g->hub_chunks + 8.0;
      int64_t cap_groups = std::max<int64_t>(1, (int64_t)(avail / per_group));
      const int64_t key_cap = (int64_t)(0xFFFFFFF0ull / (uint64_t)g->nparts);
      cap_groups = std::min<int64_t>(cap_groups, key_cap);
      nbq = std::min<int64_t>(nbq, cap_groups * Gq);
      nbq = std::min<int64_t>(nbq, nq);
    }
    const int gi = glog2 - 3;
    if (Gq == 64 && qtype == Q_SSSP && o.sched == FG_SCHED_PRIORITY && o.sched_window != 0u)
      return fail(FG_ERR_UNSUPPORTED, "the group engine has no window for groups of 64; use FIFO or a group of 32");
    if (!group_fits(g->S, Gq))
      return fail(FG_ERR_UNSUPPORTED, "group %d does not fit shared memory with partitions of %d vertices", Gq, g->S);
    if (g->group_blocks[gi] == 0)
      CUDA_TRY(group_grid_size(g->S, Gq, &g->group_blocks[gi], &g->group_threads[gi], &g->group_smem[gi]));
    const int blocks = grid_div > 1 ? std::max(1, g->group_blocks[gi] / grid_div) : g->group_blocks[gi];
    const int64_t ngroups_max = (nbq + Gq - 1) / Gq;
    const uint64_t hub_cap = (uint64_t)ngroups_max * g->hub_chunks;
    if (hub_cap + (uint64_t)ngroups_max * (uint64_t)g->nparts >= 0xFFFFFFFFull)
      return fail(FG_ERR_UNSUPPORTED, "too many work items for one launch; lower query_batch");
    CUDA_TRY(ws.g_D.reserve(4 * (size_t)ngroups_max * (size_t)npad * (size_t)Gq));
    CUDA_TRY(ws.g_pend.reserve((Gq == 64 ? 16 : 8) * (size_t)ngroups_max * (size_t)npad));
    if (qtype == Q_BFS) CUDA_TRY(ws.g_reach.reserve((Gq == 64 ? 8 : 4) * (size_t)ngroups_max * (size_t)npad));
    CUDA_TRY(ws.g_dirty.reserve(8 * (size_t)ngroups_max * (size_t)g->nparts));
    // work items, then (G = 64) the upper mask words of the hub-chunk items
    CUDA_TRY(ws.g_items.reserve(16 * (size_t)(hub_cap + (uint64_t)ngroups_max * (uint64_t)g->nparts) +
                                (Gq == 64 ? 4 * (size_t)hub_cap : 0)));
    CUDA_TRY(ws.g_best.reserve(8 * (size_t)ngroups_max));
    CUDA_TRY(ws.ctrl.reserve(sizeof(Ctrl)));
    d_ctrl = ws.ctrl.as<Ctrl>();
    CUDA_TRY(cudaMemsetAsync(d_ctrl, 0, sizeof(Ctrl), stream));
    // queries ordered by two-hop reach, so each group's (and each launch's)
    // queries advance through the graph in step; rows go back to the caller's order
    // (the rank kernel compares every pair of queries: batches up to 2^16)
    const bool reorder = o.group_order == 0 && nq > Gq && nq <= 65536;
    const int32_t *gsrc = src;
    const int32_t *rowmap = nullptr;
    if (reorder) {
      CUDA_TRY(ws.g_key.reserve(8 * (size_t)nq));
      CUDA_TRY(ws.g_perm.reserve(4 * (size_t)nq));
      CUDA_TRY(ws.g_psrc.reserve(4 * (size_t)nq));
      // graphs whose partitions keep most arcs inside (road-like): nearby
      // sources together; else sources of alike reach together
      const bool by_place = !(g->m > 0 && 2 * g->cut > g->m);
      CUDA_TRY(launch_group_order(g->dg, src, (int32_t)nq, by_place, ws.g_key.as<unsigned long long>(),
                                  ws.g_perm.as<int32_t>(),
                                  ws.g_psrc.as<int32_t>(), stream));
      launches += 2;
      gsrc = ws.g_psrc.as<int32_t>();
      rowmap = ws.g_perm.as<int32_t>();
    }
    for (int64_t q0 = 0; q0 < nq; q0 += nbq) {
      const int64_t cnt_q = std::min<int64_t>(nbq, nq - q0);
      GroupArgs a;
      a.g = g->dg;
      a.qtype = qtype;
      a.nq = (int32_t)cnt_q;
      a.G = Gq;
      a.glog2 = glog2;
      a.ngroups = (int32_t)((cnt_q + Gq - 1) / Gq);
      a.npad = npad;
      a.src = gsrc + q0;
      a.D = ws.g_D.as<uint32_t>();
      a.pend = ws.g_pend.as<uint32_t>();
      a.dirty = ws.g_dirty.as<uint32_t>();
      a.items = ws.g_items.as<uint4>();
      a.hub_cap = (uint32_t)((uint64_t)a.ngroups * g->hub_chunks);
      a.hub_hi = Gq == 64 ? reinterpret_cast<uint32_t *>(a.items + a.hub_cap + (size_t)a.ngroups * (size_t)g->nparts)
                          : nullptr;
      a.hubs = g->nhubs ? g->hubs.as<uint32_t>() : nullptr;
      a.nhubs = g->nhubs;
      a.hub_chunk = kHubChunk;
      a.window = qtype == Q_SSSP && o.sched == FG_SCHED_PRIORITY ? o.sched_window : 0u;
      a.gbest = a.window ? ws.g_best.as<uint32_t>() : nullptr;
      a.reach = qtype == Q_BFS ? ws.g_reach.as<uint32_t>() : nullptr;
      a.ctrl = d_ctrl;
      a.max_rounds = max_rounds;
      a.watchdog_ns = watchdog_ns;
      a.check_staging = o.check_staging ? 1u : 0u;
      CUDA_TRY(launch_group(a, blocks, g->group_threads[gi], g->group_smem[gi], stream));
      ++launches;
      if (rowmap) CUDA_TRY(launch_group_out(a, dist, rowmap + q0, stream));
      else CUDA_TRY(launch_group_out(a, dist + (size_t)q0 * (size_t)n, nullptr, stream));
      ++launches;
    }
  } else if (o.mode == FG_MODE_BUFFERED) {
    const uint64_t K = (uint64_t)g->nparts * (uint64_t)nb;
    // the arena holds every seed operation of a launch; beyond that a round
    // stops at 3/4 of it (arena pressure) and overflow spills losslessly into
    // the pending bitmaps. 128 slots per key (up to 2^29 slots, 20 B each)
    uint64_t e_cap = o.emit_capacity ? o.emit_capacity
                                     : std::min<uint64_t>(1ull << 29, std::max<uint64_t>(1ull << 22, 128 * K));
    e_cap = std::min<uint64_t>(std::max<uint64_t>(e_cap, (uint64_t)nb), 1ull << 31);
    if (g->engine_qtype != qtype) {
      CUDA_TRY(engine_grid_size(qtype, g->S, &g->engine_blocks, &g->engine_threads, &g->engine_smem));
      g->engine_qtype = qtype;
    }
    fg_status st = ensure_engine_ws(g, ws, qtype, nb, e_cap, need_r, g->engine_blocks);
    const int blocks = grid_div > 1 ? std::max(1, g->engine_blocks / grid_div) : g->engine_blocks;
    if (st != FG_OK) return st;
    d_ctrl = ws.ctrl.as<Ctrl>();
    CUDA_TRY(cudaMemsetAsync(d_ctrl, 0, sizeof(Ctrl), stream));
    if (!ws.pend_clean) {
      CUDA_TRY(cudaMemsetAsync(ws.pend.p, 0, ws.pend.bytes, stream));
      ws.pend_clean = true;
    }
    for (int64_t q0 = 0; q0 < nq; q0 += nb) {
      const int64_t cnt_q = std::min<int64_t>(nb, nq - q0);
      EngineArgs a;
      a.g = g->dg;
      a.qtype = qtype;
      a.nq = (int32_t)cnt_q;
      a.src = src + q0;
      const size_t row0 = (size_t)q0 * (size_t)n, rows = (size_t)cnt_q * (size_t)n;
      const bool relabelled = g->dg.orig != nullptr;
      if (qtype == Q_PPR) {
        a.pr_p = relabelled ? ws.scratch_p.as<float>() : pout + row0;
        a.pr_r = (relabelled || !rout) ? ws.scratch_r.as<float>() : rout + row0;
        a.pr_c = ws.scratch_c.as<float>();
        a.alpha = alpha;
        a.eps = eps;
      } else {
        a.dist = relabelled ? ws.state.as<uint32_t>() : dist + row0;
      }
      (void)rows;
      a.cnt = ws.cnt.as<uint32_t>();
      a.prio = ws.prio.as<uint32_t>();
      a.dirty = ws.dirty.as<uint32_t>();
      a.cur = ws.cur.as<uint32_t>();
      a.pend = ws.pend.as<uint32_t>();
      a.qbest = ws.qbest.as<uint32_t>();
      a.items = ws.items.as<uint4>();
      a.iprio = ws.iprio.as<uint32_t>();
      a.blocksum = ws.blocksum.as<unsigned long long>();
      a.e_key = ws.e_key.as<uint32_t>();
      a.e_op = ws.e_op.as<uint2>();
      a.b_op = ws.b_op.as<uint2>();
      a.e_cap = e_cap;
      a.ctrl = d_ctrl;
      a.delta = o.delta;
      a.bucket = o.bucket;
      a.sched = (uint32_t)o.sched;
      a.sched_window = o.sched_window ? o.sched_window : (o.delta ? 8u * o.delta : 0xFFFFFFFFu);
      a.yield_edges = o.yield_edges;
      a.max_rounds = max_rounds;
      a.watchdog_ns = watchdog_ns;
      // lane-per-vertex expansion only on request (measured slower than the
      // warp-shared merge-path on the road-like grid)
      a.lanes = (o.threads_per_vertex == 1 && g->max_degree <= 8) ? 1u : 0u;
      CUDA_TRY(launch_engine(a, blocks, g->engine_threads, g->engine_smem, stream));
      ++launches;
      if (qtype == Q_PPR) {
        // fold the Kahan terms, mass per query, and (if relabelled) back to original order
        if (mass && q0 == 0) CUDA_TRY(cudaMemsetAsync(mass, 0, 8 * (size_t)nq, stream));
        CUDA_TRY(launch_ppr_finalize(a, mass ? mass + q0 : nullptr, pout + row0, rout ? rout + row0 : nullptr,
                                     stream));
        ++launches;
      } else if (relabelled) {
        CUDA_TRY(launch_permute_out(a.dist, dist + row0, g->dg.orig, n, cnt_q, stream));
        ++launches;
      }
    }
  } else {
    fg_status st = ensure_plain_ws(g, ws, qtype, nb, need_r);
    if (st != FG_OK) return st;
    if (g->plain_blocks == 0) CUDA_TRY(plain_grid_size(&g->plain_blocks, &g->plain_threads));
    d_ctrl = ws.ctrl.as<Ctrl>();
    CUDA_TRY(cudaMemsetAsync(d_ctrl, 0, sizeof(Ctrl), stream));
    if (qtype == Q_PPR && mass) CUDA_TRY(cudaMemsetAsync(mass, 0, 8 * (size_t)nq, stream));
    for (int64_t q0 = 0; q0 < nq; q0 += nb) {
      const int64_t cnt_q = std::min<int64_t>(nb, nq - q0);
      for (int64_t qi = 0; qi < cnt_q; ++qi) {
        PlainArgs a;
        a.g = g->dg;
        a.qtype = qtype;
        a.q = (int32_t)(q0 + qi);
        a.nq = nq;
        a.src = src;
        const size_t row = (size_t)(q0 + qi) * (size_t)n;
        if (qtype == Q_PPR) {
          a.out_p = pout + row;
          a.out_r = rout ? rout + row : ws.scratch_r.as<float>() + (size_t)qi * (size_t)n;
          a.out_c = ws.scratch_c.as<float>() + (size_t)qi * (size_t)n;
          a.rr = ws.pl_rr.as<float>();
          a.pp = ws.pl_pp.as<float>();
          a.cc = ws.pl_cc.as<float>();
        } else {
          a.out_u32 = dist + row;
          a.dist = ws.pl_dist.as<uint32_t>();
        }
        a.stamp = ws.pl_stamp.as<uint32_t>();
        a.front[0] = ws.pl_f0.as<uint32_t>();
        a.front[1] = ws.pl_f1.as<uint32_t>();
        a.sizes = ws.pl_sizes.as<uint32_t>();
        a.alpha = alpha;
        a.eps = eps;
        a.max_rounds = max_rounds;
        a.watchdog_ns = watchdog_ns;
        a.ctrl = d_ctrl;
        CUDA_TRY(launch_plain(a, g->plain_blocks, g->plain_threads, stream));
        ++launches;
      }
      if (qtype == Q_PPR) {
        // the plain kernel already wrote original order: fold in place
        EngineArgs f;
        f.g = g->dg;
        f.g.orig = nullptr;
        f.nq = (int32_t)cnt_q;
        f.pr_p = pout + (size_t)q0 * (size_t)n;
        f.pr_r = rout ? rout + (size_t)q0 * (size_t)n : ws.scratch_r.as<float>();
        f.pr_c = ws.scratch_c.as<float>();
        CUDA_TRY(launch_ppr_finalize(f, mass ? mass + q0 : nullptr, f.pr_p, rout ? f.pr_r : nullptr, stream));
        ++launches;
      }
    }
  }
  if (shared_ws) {
    CUDA_TRY(cudaEventRecord(g->last_done, stream));
    g->has_last = true;
  }

  // status and statistics travel back with the stream
  Ctrl *h = take_slot();
  if (!h) return fail(FG_ERR_OOM, "pinned status slot allocation failed");
  std::memset(h, 0, sizeof(Ctrl));
  cudaError_t ce = cudaMemcpyAsync(h, d_ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, stream);
  if (ce != cudaSuccess) {
    std::lock_guard<std::mutex> lp(g_pending_mu);
    g_slot_pool.push_back(h);
    return fail(FG_ERR_CUDA, "status copy: %s", cudaGetErrorString(ce));
  }
  {
    std::lock_guard<std::mutex> lp(g_pending_mu);
    g_pending.push_back(Pending{stream, g, &ws, h, (unsigned)launches, (unsigned)Gq});
  }
  if (host_io) {
    if (qtype == Q_PPR) {
      CUDA_TRY(cudaMemcpyAsync(p_in, pout, 4 * row_elems, cudaMemcpyDeviceToHost, stream));
      if (r_in) CUDA_TRY(cudaMemcpyAsync(r_in, rout, 4 * row_elems, cudaMemcpyDeviceToHost, stream));
      if (mass_in) CUDA_TRY(cudaMemcpyAsync(mass_in, mass, 8 * (size_t)nq, cudaMemcpyDeviceToHost, stream));
    } else {
      CUDA_TRY(cudaMemcpyAsync(dist_in, dist, 4 * row_elems, cudaMemcpyDeviceToHost, stream));
    }
    CUDA_TRY(cudaEventRecord(io->done, stream));
    io->used = true;
    if (o.host_io == 1) CUDA_TRY(cudaStreamSynchronize(stream));
  }
  return FG_OK;
}

}  // namespace fg

namespace {

fg_status run_batch(fg_graph *g, int qtype, const int32_t *src_in, int32_t nq, uint32_t *dist_in, float alpha,
                    float eps, float *p_in, float *r_in, double *mass_in, void *stream_v, const fg_opts *opts_in) {
  if (!g) return fail(FG_ERR_INVALID_ARG, "graph is NULL");
  return run_batch_on(g, g->ws, true, 1, qtype, src_in, nq, dist_in, alpha, eps, p_in, r_in, mass_in, stream_v,
                      opts_in);
}

}  // namespace

extern "C" fg_status fg_sssp_batch(fg_graph *g, const int32_t *src, int32_t nq, uint32_t *dist_out, void *stream,
                                   const fg_opts *opts) {
  return run_batch(g, Q_SSSP, src, nq, dist_out, 0.f, 0.f, nullptr, nullptr, nullptr, stream, opts);
}

extern "C" fg_status fg_bfs_batch(fg_graph *g, const int32_t *src, int32_t nq, uint32_t *level_out, void *stream,
                                  const fg_opts *opts) {
  return run_batch(g, Q_BFS, src, nq, level_out, 0.f, 0.f, nullptr, nullptr, nullptr, stream, opts);
}

extern "C" fg_status fg_ppr_batch(fg_graph *g, const int32_t *src, int32_t nq, float alpha, float eps, float *p_out,
                                  float *r_out, double *mass_out, void *stream, const fg_opts *opts) {
  return run_batch(g, Q_PPR, src, nq, nullptr, alpha, eps, p_out, r_out, mass_out, stream, opts);
}

extern "C" fg_status fg_sync(void *stream_v) {
  cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_v);
  cudaError_t e = cudaStreamSynchronize(stream);
  std::vector<Pending> mine;
  {
    std::lock_guard<std::mutex> lp(g_pending_mu);
    for (size_t i = 0; i < g_pending.size();) {
      if (g_pending[i].stream == stream) {
        mine.push_back(g_pending[i]);
        g_pending[i] = g_pending.back();
        g_pending.pop_back();
      } else {
        ++i;
      }
    }
  }
  fg_status first = FG_OK;
  if (e != cudaSuccess) first = fail(FG_ERR_CUDA, "cudaStreamSynchronize: %s", cudaGetErrorString(e));
  for (Pending &p : mine) {
    const Ctrl &c = *p.host;
    if (p.graph) {
      fg_stats_t s{};
      s.rounds = c.rounds;
      s.visits = c.visits;
      s.edges = c.edges;
      s.ops = c.ops;
      s.spills = c.spills;
      s.yields = c.yields;
      s.launches = p.launches;
      s.max_round_ops = c.max_round_ops;
      for (int k = 0; k < 6; ++k) s.phase_ns[k] = c.phase_ns[k];
      s.arcs_read = c.arcs_read;
      s.group = p.group;
      p.graph->last_stats = s;
      if (c.status != 0 && c.status != FG_ERR_OVERFLOW && p.ws) p.ws->pend_clean = false;
    }
    if (first == FG_OK && c.status != 0) {
      const char *names[] = {"ok", "invalid argument", "out of memory", "CUDA error", "watchdog timeout",
                             "operation buffer overflow", "distance overflow", "unsupported"};
      const char *sites[] = {"", " (device-wide barrier wait)", " (shared-memory staging wait)",
                             " (visit step limit)", " (max_rounds)", " (source id out of range)",
                             " (operation arena)", " (vertex degree out of range)", " (work-item claim wait)",
                             " (staged words differ from global memory)"};
      const int k = c.status >= 0 && c.status <= 7 ? c.status : 3;
      const unsigned si = c.site <= 9 ? c.site : 0;
      first = fail((fg_status)c.status, "device reported: %s%s", names[k], sites[si]);
    }
    std::lock_guard<std::mutex> lp(g_pending_mu);
    g_slot_pool.push_back(p.host);
  }
  return first;
}

namespace fg {

int auto_group_size(const fg_graph *g, int qtype, int64_t nq, bool windowed) {
  if (!(g->m > 0 && 2 * g->cut > g->m)) return 1;
  int G = (qtype == Q_BFS || windowed) ? 32 : 64;  // groups of 64 run FIFO rounds only
  while (G > 8 && (int64_t)(G / 2) >= nq) G /= 2;  // a small batch: the smallest group that holds it
  while (G > 8 && !group_fits(g->S, G)) G /= 2;
  return group_fits(g->S, G) ? G : 1;
}

fg_status report_error(fg_status s, const char *msg) {
  t_err = msg ? msg : "";
  return s;
}

void graph_device_view(const fg_graph *g, DevGraph *dg, int *device) {
  *dg = g->dg;
  *device = g->device;
}

}  // namespace fg
