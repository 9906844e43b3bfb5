// Internal structures shared by the host runtime and the CUDA kernels.
#pragma once

#include <cstdint>

#include <cuda_runtime.h>

#include "../../include/fg.h"

namespace fg {

enum QType : int { Q_SSSP = 0, Q_BFS = 1, Q_PPR = 2 };

constexpr uint32_t kInf = 0xFFFFFFFFu;
constexpr uint32_t kInvalidKey = 0xFFFFFFFFu;

// where a device status was raised (reported by fg_sync)
enum : unsigned { kSiteNone = 0, kSiteBarrier = 1, kSiteStage = 2, kSiteVisit = 3, kSiteRounds = 4,
                  kSiteSource = 5, kSiteArena = 6, kSiteDegree = 7, kSiteClaim = 8, kSiteStageCheck = 9 };

// Graph in partition-major ("internal") vertex order. Partition j holds the
// internal ids [j*S, (j+1)*S); S = 1 << slog2.
struct DevGraph {
  int32_t n = 0;
  int32_t slog2 = 0;
  int32_t S = 0;
  int32_t nparts = 0;
  uint64_t m = 0;
  uint32_t max_deg = 0;            // largest out-degree (bounds every arc loop)
  uint32_t max_w = 1;              // largest arc weight (1 when unweighted)
  const uint32_t *rp = nullptr;    // [n+1] arc offsets
  const uint32_t *adj = nullptr;   // [m] internal target ids
  const uint32_t *wt = nullptr;    // [m] weights, or null (unit)
  const int32_t *orig = nullptr;   // [n] internal -> original id, or null (identity)
  const int32_t *intl = nullptr;   // [n] original -> internal id, or null (identity)
};

// Device control block of one batch launch (zeroed before each launch).
struct Ctrl {
  unsigned int bar_count;
  unsigned int bar_gen;
  int status;                 // fg_status raised on the device (0 = ok)
  int abort;                  // set with status: every block leaves at its next check
  unsigned int item_next;     // work-claiming counter of the current round
  unsigned int site;          // where the first status was raised (kSite*)
  unsigned long long e_cursor;  // operations reserved in the arena this round
  unsigned long long rounds, visits, edges, ops, spills, yields, max_round_ops;
  unsigned long long phase_ns[6];  // K0, INIT, SCAN-A, SCAN-B, SCATTER, PROCESS (block 0's view)
  // group engine: per round parity, the items found by the scan (hub chunks,
  // partition items) and the claiming counter
  unsigned int g_hub_items[2], g_items[2], g_next[2];
  unsigned long long arcs_read;  // graph arcs read (per query visit, or per group visit)
  unsigned int max_ops[2];       // largest buffer of the round, per round parity (max-operations scheduling)
  unsigned int g_exit;           // group engine, serve mode: the launch ends after this round
};

// Serve mode of the group engine (continuous batching): a mailbox in mapped
// host memory. The host writes a slot's source, then a new sequence number;
// at a round boundary the running launch admits it into that query lane and
// acknowledges it; when the lane's query has no pending work left, the launch
// copies its row out and writes the sequence number to done_seq.
struct ServeSlot {
  int32_t src;        // host: original source id
  uint32_t seq;       // host: a new value = a new request in this slot
  uint32_t ack;       // device: the last sequence number admitted
  uint32_t done_seq;  // device: the last sequence number completed (its row is in res)
  int32_t status;     // device: fg_status of that request
  uint32_t pad[3];
};
struct ServeBox {
  uint32_t stop;      // host: leave at the next round boundary, work or not (the state is then refilled)
  uint32_t pad[7];
  ServeSlot slot[1];  // [slots]
};

struct EngineArgs {
  DevGraph g;
  int qtype = Q_SSSP;
  int32_t nq = 0;
  const int32_t *src = nullptr;   // [nq] original ids (device)
  // query state, query-major [nq][n], internal (partition-major) vertex order
  uint32_t *dist = nullptr;       // SSSP / BFS
  float *pr_p = nullptr;          // PPR estimate
  float *pr_r = nullptr;          // PPR residual
  float *pr_c = nullptr;          // PPR Kahan compensation
  float alpha = 0.f, eps = 0.f;
  // per-(partition, query) buffers, key = p * nq + q
  uint32_t *cnt = nullptr;        // [K] operations buffered this round
  uint32_t *prio = nullptr;       // [K] best pending value (SSSP/BFS)
  uint32_t *dirty = nullptr;      // [K] pending bitmap non-empty
  uint32_t *cur = nullptr;        // [K] scatter cursor
  uint32_t *pend = nullptr;       // [K][S/32] deferred vertices
  uint32_t *qbest = nullptr;      // [nq] best pending value per query (priority scheduling)
  uint4 *items = nullptr;         // [K] {key, offset, count, flags}
  uint32_t *iprio = nullptr;      // [K] best value of each work item (priority carry-over)
  unsigned long long *blocksum = nullptr;  // [2 * grid]: (ops << 32 | items) per block, then items with pending vertices
  // operation arena (append order) and bins (key order)
  uint32_t *e_key = nullptr;
  uint2 *e_op = nullptr;
  uint2 *b_op = nullptr;
  uint64_t e_cap = 0;
  Ctrl *ctrl = nullptr;
  // options
  uint32_t delta = 0, bucket = 0, sched = 0, sched_window = 0;
  uint64_t yield_edges = 0;
  uint32_t max_rounds = 0;
  uint64_t watchdog_ns = 0;
  uint32_t lanes = 0;  // 1: lane-per-vertex expansion (max out-degree <= 8)
};

// Group engine (fg_group.cu): G queries per group, lanes = queries. State is
// vertex-major inside a group, D[group][vertex][G] in internal order, so the
// G values of one vertex are one contiguous line. A vertex whose value was
// lowered in round r is marked in pend[(r + 1) & 1][group][vertex] (a mask of
// G bits) and its partition in dirty[(r + 1) & 1][group * nparts + p].
struct GroupArgs {
  DevGraph g;
  int qtype = Q_SSSP;
  int32_t nq = 0;
  int32_t G = 16;                 // queries per group: 8, 16, 32 or 64
  int32_t glog2 = 4;              // log2(G)
  int32_t ngroups = 0;            // ceil(nq / G)
  int64_t npad = 0;               // nparts * S: vertices per group row, padded to whole partitions
  const int32_t *src = nullptr;   // [nq] original ids (device)
  uint32_t *D = nullptr;          // [ngroups][npad][G]
  uint32_t *pend = nullptr;       // [2][ngroups][npad] G-bit masks (32-bit words; 64-bit for G = 64)
  uint32_t *dirty = nullptr;      // [2][ngroups * nparts]
  uint4 *items = nullptr;         // [hub_cap + ngroups * nparts]
  uint32_t *hub_hi = nullptr;     // [hub_cap] G = 64: upper mask word of each hub-chunk item
  uint32_t hub_cap = 0;           // item slots reserved for hub chunks
  const uint32_t *hubs = nullptr; // [nhubs] internal ids of the hubs (vertices with many arcs)
  int32_t nhubs = 0;
  uint32_t hub_chunk = 4096;      // arcs per hub chunk (a work item of its own)
  uint32_t window = 0;            // per-group value window of a round (0 = none)
  uint32_t *gbest = nullptr;      // [2][ngroups] smallest pending value per group (window scheduling)
  uint32_t *reach = nullptr;      // BFS: [ngroups][npad] G-bit masks of the queries that reached each vertex
  uint32_t *lstart = nullptr;     // BFS in serve mode: [slots] the round each lane's query started
  Ctrl *ctrl = nullptr;
  uint32_t max_rounds = 0;
  uint64_t watchdog_ns = 0;
  // serve mode (continuous batching); off when box is null
  ServeBox *box = nullptr;        // mapped host mailbox, ngroups * G slots (device address)
  uint32_t *res = nullptr;        // [slots][n] result rows, original vertex order
  uint32_t *occ = nullptr;        // [ngroups] lanes holding an admitted, unfinished query
  uint32_t *seen = nullptr;       // [slots] sequence number of each slot's current request
  uint32_t *gact = nullptr;       // [2][ngroups] lanes with pending work in the round of that parity
  uint32_t check_staging = 0;     // 1: compare every staged word with global memory (self-test)
  uint32_t init = 0;              // 1: first launch on this state: fill it before the first round
  uint32_t round0 = 0;            // number of the first round (its parity selects the mask halves)
};

struct PlainArgs {
  DevGraph g;
  int qtype = Q_SSSP;
  int32_t q = 0;
  int32_t nq = 0;
  uint32_t *out_u32 = nullptr;    // row base of query q (original order)
  const int32_t *src = nullptr;   // [nq] original source ids (device)
  float *out_p = nullptr, *out_r = nullptr, *out_c = nullptr;  // row bases (original order)
  uint32_t *dist = nullptr;       // [n] scratch, internal order
  float *rr = nullptr, *pp = nullptr, *cc = nullptr;  // [n] scratch, internal order
  uint32_t *stamp = nullptr;      // [n]
  uint32_t *front[2] = {nullptr, nullptr};  // [n] each
  uint32_t *sizes = nullptr;      // [3]
  float alpha = 0.f, eps = 0.f;
  uint32_t max_rounds = 0;
  uint64_t watchdog_ns = 0;
  Ctrl *ctrl = nullptr;
};

// kernel launchers (fg_engine.cu / fg_plain.cu); return the CUDA error of the launch
cudaError_t engine_grid_size(int qtype, int S, int *blocks, int *threads, size_t *smem);
cudaError_t launch_engine(const EngineArgs &a, int blocks, int threads, size_t smem, cudaStream_t s);
cudaError_t launch_ppr_finalize(const EngineArgs &a, double *mass, float *p_out, float *r_out, cudaStream_t s);
cudaError_t launch_permute_out(const uint32_t *state, uint32_t *out, const int32_t *orig, int64_t n, int64_t rows,
                               cudaStream_t s);
cudaError_t plain_grid_size(int *blocks, int *threads);
// Whether a group-engine block for partitions of S vertices and groups of G
// fits the device's shared memory per block.
bool group_fits(int S, int G);
cudaError_t group_grid_size(int S, int G, int *blocks, int *threads, size_t *smem);
cudaError_t launch_group(const GroupArgs &a, int blocks, int threads, size_t smem, cudaStream_t s);
// Orders a batch's queries for the group engine: key[q] = arcs within two hops
// of src[q], or (by_place) the source's internal id counted down; perm[j] =
// the query in slot j (keys descending, ties by index), psrc[j] =
// src[perm[j]]. key, perm and psrc hold nq entries each.
cudaError_t launch_group_order(const DevGraph &g, const int32_t *src, int32_t nq, bool by_place,
                               unsigned long long *key, int32_t *perm, int32_t *psrc, cudaStream_t s);
// group-engine state (internal order, vertex-major in groups) -> caller's query-major rows
// Writes the launch's rows to out: slot j's row to out[rowmap[j] * n], or to
// out[j * n] when rowmap is null.
cudaError_t launch_group_out(const GroupArgs &a, uint32_t *out, const int32_t *rowmap, cudaStream_t s);
cudaError_t launch_plain(const PlainArgs &a, int blocks, int threads, cudaStream_t s);

// runtime services for entry points outside fg_runtime.cpp
fg_status report_error(fg_status s, const char *msg);  // sets fg_last_error(), returns s
void graph_device_view(const fg_graph *g, DevGraph *dg, int *device);
// set-up of fg_sssp_batch_noalloc's fixed scratch on device dev (current); best effort
void noalloc_prepare(int dev);

}  // namespace fg
