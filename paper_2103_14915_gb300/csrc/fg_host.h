// Host-side structures shared by the runtime (fg_runtime.cpp) and the
// serving loop (fg_server.cpp): device buffers, per-batch workspace, the
// graph handle and the batch launcher.
#pragma once

#include <cstddef>
#include <cstdint>
#include <map>
#include <mutex>
#include <utility>

#include "fg_internal.h"

namespace fg {

// Sets the calling thread's fg_last_error() message (printf format) and returns s.
fg_status fail(fg_status s, const char *fmt, ...);

#define CUDA_TRY(expr)                                                                      \
  do {                                                                                      \
    cudaError_t e_ = (expr);                                                                \
    if (e_ != cudaSuccess)                                                                  \
      return fail(e_ == cudaErrorMemoryAllocation ? FG_ERR_OOM : FG_ERR_CUDA, "%s: %s (%s:%d)", \
                  #expr, cudaGetErrorString(e_), __FILE__, __LINE__);                       \
  } while (0)

struct DevBuf {
  void *p = nullptr;
  size_t bytes = 0;
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
  }
  cudaError_t reserve(size_t b) {
    if (b <= bytes && p) return cudaSuccess;
    release();
    cudaError_t e = cudaMalloc(&p, b ? b : 16);
    if (e == cudaSuccess) bytes = b;
    else p = nullptr;
    return e;
  }
  template <typename T>
  T *as() const { return reinterpret_cast<T *>(p); }
};

// Device staging of one host-I/O batch (sources, outputs). A workspace keeps
// two, used in turn, so that one batch's copy to the host can overlap the next
// batch's kernels; `done` is recorded after a slot's copy to the host.
struct IoSlot {
  DevBuf src, out, out2;
  cudaEvent_t done = nullptr;
  bool used = false;
  void release() {
    src.release();
    out.release();
    out2.release();
    if (done) cudaEventDestroy(done);
    done = nullptr;
    used = false;
  }
};

struct Workspace {
  DevBuf cnt, prio, dirty, cur, pend, qbest, items, iprio, blocksum, e_key, e_op, b_op, ctrl;
  DevBuf g_D, g_pend, g_dirty, g_items, g_best, g_reach;  // group engine
  DevBuf g_key, g_perm, g_psrc;                   // group engine: query order (two-hop reach)
  DevBuf scratch_r, scratch_c, scratch_p, state;
  DevBuf pl_dist, pl_rr, pl_pp, pl_cc, pl_stamp, pl_f0, pl_f1, pl_sizes;
  IoSlot io[2];
  int io_next = 0;
  bool pend_clean = true;
  void release_all() {
    DevBuf *all[] = {&cnt, &prio, &dirty, &cur, &pend, &qbest, &items, &iprio, &blocksum, &e_key, &e_op,
                     &b_op, &ctrl, &scratch_r, &scratch_c, &scratch_p, &state, &pl_dist, &pl_rr,
                     &pl_pp, &pl_cc, &pl_stamp, &pl_f0, &pl_f1, &pl_sizes, &g_D, &g_pend, &g_dirty, &g_reach,
                     &g_items, &g_best, &g_key, &g_perm, &g_psrc};
    for (DevBuf *b : all) b->release();
    io[0].release();
    io[1].release();
  }
};

// Scratch of fg_bc_accumulate, grown on demand and kept with the graph.
struct BcWorkspace {
  DevBuf pc, sigma, delta, dint, wave, wave_off, ctrl;
  void release_all() {
    DevBuf *all[] = {&pc, &sigma, &delta, &dint, &wave, &wave_off, &ctrl};
    for (DevBuf *b : all) b->release();
  }
};

// Scratch of fg_dfs_batch: per query a stack of (vertex, arc to resume from),
// a bitmap of discovered vertices and, for a relabelled graph, the discovery
// ranks in internal order.
struct DfsWorkspace {
  DevBuf stack, disc, flag, seen;
  void release_all() {
    stack.release();
    disc.release();
    flag.release();
    seen.release();
  }
};

struct TuneKey {
  int kind, bucket;
  uint32_t alpha_bits, eps_bits;
  bool operator<(const TuneKey &o) const {
    if (kind != o.kind) return kind < o.kind;
    if (bucket != o.bucket) return bucket < o.bucket;
    if (alpha_bits != o.alpha_bits) return alpha_bits < o.alpha_bits;
    return eps_bits < o.eps_bits;
  }
};

}  // namespace fg

// Graph handle of the C ABI: the partitioned graph on the device, its own
// batch workspace, and the cached launch shapes.
struct fg_graph {
  fg::DevGraph dg;
  int64_t n = 0, m = 0;
  int method = FG_PART_RANGE, S = 0, slog2 = 0, nparts = 0;
  int64_t cut = 0;
  bool weighted = false;
  int device = 0;
  fg::DevBuf rp, adj, wt, orig, intl;
  fg::DevBuf deg;                  // out-degree per original id (built by the first fg_ncp_sweep)
  fg::BcWorkspace bc;              // fg_bc_accumulate scratch (guarded by mu)
  fg::DfsWorkspace dfs;            // fg_dfs_batch scratch (guarded by mu)
  bool has_zero_weight = false;    // some arc has weight 0
  int bc_blocks = 0;               // cooperative grid of the BC kernel (0 = not sized yet)
  size_t graph_bytes = 0;
  std::mutex mu;                   // guards ws, last_done and the cached launch shapes
  cudaEvent_t last_done = nullptr;
  bool has_last = false;
  fg::Workspace ws;
  fg_stats_t last_stats{};
  int engine_blocks = 0, engine_threads = 0;
  size_t engine_smem = 0;
  int engine_qtype = -1;
  uint32_t max_degree = 0;
  double mean_weight = 1.0;        // mean arc weight (1 when unweighted)
  uint32_t max_weight = 0;         // largest arc weight (0 when unweighted)
  // choices of fg_tune_opts[_ex], keyed by (query kind, log2 of the batch size
  // rounded up, and for PPR the bits of alpha and eps)
  std::map<fg::TuneKey, std::pair<fg_opts, fg_tune_report>> tuned;
  int plain_blocks = 0, plain_threads = 0;
  // group engine: the hubs, vertices with more than kHubMin arcs (internal ids),
  // relaxed in chunks of at most kHubChunk arcs spread over blocks, and the
  // number of chunks they make; launch shapes per group size (index log2(G) - 3)
  fg::DevBuf hubs;
  int32_t nhubs = 0;
  uint64_t hub_chunks = 0;
  int group_blocks[4] = {0, 0, 0, 0}, group_threads[4] = {0, 0, 0, 0};
  size_t group_smem[4] = {0, 0, 0, 0};
};

namespace fg {

constexpr uint32_t kHubMin = 512;     // group engine: vertices with more arcs are hubs
constexpr uint32_t kHubChunk = 4096;  // group engine: arcs per hub chunk

// The query group that fg_opts.group = 0 resolves to for a batch of nq
// queries of one kind: on graphs whose partitions are cut by more than half
// of the arcs, 64 for SSSP (32 under a window) and 32 for BFS (the smallest of
// 8, 16, 32, 64 that holds a smaller batch, and one that fits shared memory);
// else 1.
int auto_group_size(const fg_graph *g, int qtype, int64_t nq, bool windowed);

// One batch of nq queries on workspace ws (see fg_runtime.cpp).
fg_status run_batch_on(fg_graph *g, Workspace &ws, bool shared_ws, int grid_div, int qtype, const int32_t *src_in,
                       int32_t nq, uint32_t *dist_in, float alpha, float eps, float *p_in, float *r_in,
                       double *mass_in, void *stream_v, const fg_opts *opts_in);

}  // namespace fg
