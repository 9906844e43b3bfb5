// Betweenness centrality from sampled sources: the BC application, which runs
// one SSSP (weighted graph) or BFS (unweighted graph) per sampled source and
// gathers the results into centralities (Sec. 1; Sec. 6.1 samples 100
// sources), with the dependency accumulation of Brandes that the paper cites.
//
// Input: the batch's exact distance rows (fg_sssp_batch / fg_bfs_batch
// output). An arc (u, w) is tight for source s when d(u) + wt(u, w) = d(w);
// the tight arcs form the shortest-path DAG of s. Per source:
//   count    tight in-arcs per vertex (atomics over every reachable vertex's
//            out-arcs);
//   forward  topological waves over the DAGs: wave 0 holds the sources; a
//            vertex of wave t adds its path count sigma to each tight
//            successor and releases it into wave t + 1 when the successor's
//            last tight in-arc is done. Path counts are integers, so the FP64
//            atomic sums are exact in any order while they stay below 2^53
//            (the call reports when one reaches it);
//   backward waves in reverse order: delta(u) = sum over u's tight out-arcs in
//            CSR order of sigma(u) / sigma(w) * (1 + delta(w)), each operation
//            rounded as written (no fused multiply-add);
//   gather   bc(v) += delta_s(v) over the sources s != v, in batch order.
// Two forms run these steps. bc_kernel is one cooperative launch over all the
// batch's sources: their waves advance together, separated by device-wide
// barriers (bounded waits), which suits shallow, wide DAGs (social graphs).
// bc_block_kernel runs one source per block with the block's own barrier
// between waves, which suits the deep, narrow DAGs of road-like graphs
// (thousands of waves), and bc_gather_kernel does the gather afterwards.
#include <algorithm>
#include <cstdint>
#include <cstdio>
#include <cstring>

#include "fg_device.cuh"
#include "fg_host.h"

namespace fg {
namespace {

constexpr int kBcThreads = 256;
constexpr uint32_t kRoadDegree = 64;  // max out-degree up to which a graph takes one block per source
constexpr double kExactLimit = 9007199254740992.0;  // 2^53

// Counters of one launch (zeroed before it). Wave t appends the vertices it
// releases through cnt[(t + 1) % 3]; everyone reads that count after the
// barrier that ends wave t, and the counter wave t + 1 appends through is
// cleared during wave t, when its previous count has been read by all.
struct BcCounters {
  unsigned long long cnt[3];
  unsigned long long waves;
  unsigned long long inexact;     // a path count reached 2^53
  unsigned long long sigma_max;   // bit pattern of the largest path count (non-negative double)
};

struct BcArgs {
  DevGraph g;                 // internal (partition-major) order
  int32_t nq = 0;
  const int32_t *src = nullptr;     // [nq] original ids
  const uint32_t *dist = nullptr;   // [nq][n] original order
  uint32_t *dint = nullptr;         // [nq][n] the same rows in internal order (null: identity order)
  bool weighted = false;
  uint32_t *pc = nullptr;           // [nq][n] tight in-arcs not yet done (internal order)
  double *sigma = nullptr;          // [nq][n] shortest-path counts
  double *delta = nullptr;          // [nq][n] dependencies
  uint2 *wave = nullptr;            // [nq * n] (query, vertex) in wave order
  uint32_t *wave_off = nullptr;     // [n + 2] first entry of each wave
  double *bc = nullptr;             // [n] original order
  bool accumulate = false;
  Ctrl *ctrl = nullptr;             // device-wide barrier and status
  BcCounters *cn = nullptr;
  uint64_t watchdog_ns = 0;
};

// d_q(u) for an internal vertex id (rows written by this launch: read through L2)
__device__ __forceinline__ uint32_t dist_of(const BcArgs &a, int64_t q, uint32_t u) {
  const int64_t i = q * (int64_t)a.g.n + u;
  return a.dint ? __ldcg(a.dint + i) : __ldg(a.dist + i);
}

__device__ __forceinline__ bool tight(uint32_t du, uint32_t wt, uint32_t dw) {
  return dw != kInf && (uint64_t)du + (uint64_t)wt == (uint64_t)dw;
}

constexpr uint32_t kLight = 32;  // out-degree up to which one lane handles a vertex; above, the whole warp

struct Item {
  int64_t q;
  uint32_t u, e0, e1;
};

// Warp-centric walk over items [0, count): lane i of a warp takes item
// base + i; a light item is handled by its lane (`lane_fn`), heavy items are
// then handled one after another by the whole warp (`warp_fn`, lanes striding
// the arcs). `item_at(i)` yields the (query, vertex) of item i.
template <class ItemAt, class LaneFn, class WarpFn>
__device__ __forceinline__ void walk_items(int64_t count, ItemAt item_at, LaneFn lane_fn, WarpFn warp_fn,
                                           const DevGraph &g) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t base = warp * 32; base < count; base += nwarps * 32) {
    const int64_t i = base + lane;
    Item it{0, 0, 0, 0};
    const bool valid = i < count;
    if (valid) {
      item_at(i, it.q, it.u);
      it.e0 = __ldg(g.rp + it.u);
      it.e1 = __ldg(g.rp + it.u + 1);
    }
    const bool light = valid && it.e1 - it.e0 <= kLight;
    if (light) lane_fn(it);
    unsigned heavy = __ballot_sync(kFull, valid && !light);
    while (heavy) {
      const int j = __ffs(heavy) - 1;
      heavy &= heavy - 1;
      Item h;
      h.q = __shfl_sync(kFull, it.q, j);
      h.u = __shfl_sync(kFull, it.u, j);
      h.e0 = __shfl_sync(kFull, it.e0, j);
      h.e1 = __shfl_sync(kFull, it.e1, j);
      warp_fn(h, lane);
    }
  }
}

// Append (q, w) to the next wave; lanes that release at the same time share
// one atomic on the wave's counter.
__device__ __forceinline__ void release(const BcArgs &a, unsigned long long *appends, uint32_t end, int64_t total,
                                        int64_t q, uint32_t w) {
  const unsigned m = __activemask();
  const int lane = threadIdx.x & 31;
  const int leader = __ffs(m) - 1;
  unsigned long long base = 0;
  if (lane == leader) base = atomicAdd(appends, (unsigned long long)__popc(m));
  base = __shfl_sync(m, base, leader);
  const unsigned long long pos = (unsigned long long)end + base + (unsigned long long)__popc(m & ((1u << lane) - 1u));
  if (pos < (unsigned long long)total) a.wave[pos] = make_uint2((uint32_t)q, w);
  else raise_status(a.ctrl, FG_ERR_INVALID_ARG, kSiteArena);  // cannot happen: each vertex is released once
}

// sigma(u) / sigma(w) * (1 + delta(w)) for a tight arc, each operation rounded as written
__device__ __forceinline__ double dep_term(double su, double sw, double dw) {
  return __dmul_rn(__ddiv_rn(su, sw), __dadd_rn(1.0, dw));
}

__global__ void __launch_bounds__(kBcThreads) bc_kernel(BcArgs a) {
  const int64_t n = a.g.n;
  const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
  const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t total = (int64_t)a.nq * n;
  const int lane = threadIdx.x & 31;
  unsigned gen = 0;

  // ---- init -------------------------------------------------------------
  for (int64_t i = gtid; i < total; i += nthreads) {
    a.pc[i] = 0u;
    a.sigma[i] = 0.0;
    a.delta[i] = 0.0;
    if (a.dint) {
      const int64_t q = i / n, u = i - q * n;
      a.dint[i] = __ldg(a.dist + q * n + __ldg(a.g.orig + u));
    }
  }
  for (int64_t q = gtid; q < a.nq; q += nthreads) {
    const int32_t s = a.src[q];
    if (s < 0 || (int64_t)s >= n || __ldg(a.dist + q * n + s) != 0u) raise_status(a.ctrl, FG_ERR_INVALID_ARG, kSiteSource);
  }
  if (!grid_barrier(a.ctrl, gen, a.watchdog_ns)) return;
  for (int64_t q = gtid; q < a.nq; q += nthreads) {
    const uint32_t s = a.g.intl ? (uint32_t)a.g.intl[a.src[q]] : (uint32_t)a.src[q];
    a.sigma[q * n + s] = 1.0;
    a.wave[q] = make_uint2((uint32_t)q, s);
  }
  if (gtid == 0) a.wave_off[0] = 0u;

  // ---- count tight in-arcs ------------------------------------------------
  auto all_items = [n](int64_t i, int64_t &q, uint32_t &u) {
    q = i / n;
    u = (uint32_t)(i - q * n);
  };
  walk_items(
      total, all_items,
      [&](const Item &it) {
        const uint32_t du = dist_of(a, it.q, it.u);
        if (du == kInf) return;
        for (uint32_t e = it.e0; e < it.e1; ++e) {
          const uint32_t w = __ldg(a.g.adj + e);
          const uint32_t wt = a.weighted ? __ldg(a.g.wt + e) : 1u;
          if (tight(du, wt, dist_of(a, it.q, w))) atomicAdd(a.pc + it.q * n + w, 1u);
        }
      },
      [&](const Item &it, int ln) {
        const uint32_t du = dist_of(a, it.q, it.u);
        if (du == kInf) return;
        for (uint32_t e = it.e0 + ln; e < it.e1; e += 32) {
          const uint32_t w = __ldg(a.g.adj + e);
          const uint32_t wt = a.weighted ? __ldg(a.g.wt + e) : 1u;
          if (tight(du, wt, dist_of(a, it.q, w))) atomicAdd(a.pc + it.q * n + w, 1u);
        }
      },
      a.g);
  if (!grid_barrier(a.ctrl, gen, a.watchdog_ns)) return;

  // ---- forward waves: path counts --------------------------------------------
  double smax = 0.0;  // this lane's largest path count seen
  uint32_t beg = 0, count = (uint32_t)a.nq, waves = 0;
  while (count > 0) {
    const uint32_t end = beg + count;
    unsigned long long *appends = &a.cn->cnt[(waves + 1) % 3];
    if (gtid == 0) {
      a.cn->cnt[(waves + 2) % 3] = 0ull;  // wave t + 1 appends through it; its last count was read a wave ago
      a.wave_off[waves + 1] = end;
    }
    auto wave_items = [&](int64_t i, int64_t &q, uint32_t &u) {
      const uint2 it = __ldcg(a.wave + beg + i);
      q = it.x;
      u = it.y;
    };
    auto push = [&](const Item &it, uint32_t e, double su, uint32_t du) {
      const uint32_t w = __ldg(a.g.adj + e);
      const uint32_t wt = a.weighted ? __ldg(a.g.wt + e) : 1u;
      if (!tight(du, wt, dist_of(a, it.q, w))) return;
      const double now = atomicAdd(a.sigma + it.q * n + w, su) + su;
      smax = now > smax ? now : smax;
      if (atomicSub(a.pc + it.q * n + w, 1u) == 1u) release(a, appends, end, total, it.q, w);  // last tight in-arc
    };
    walk_items(
        (int64_t)count, wave_items,
        [&](const Item &it) {
          const double su = __ldcg(a.sigma + it.q * n + it.u);
          const uint32_t du = dist_of(a, it.q, it.u);
          for (uint32_t e = it.e0; e < it.e1; ++e) push(it, e, su, du);
        },
        [&](const Item &it, int ln) {
          const double su = __ldcg(a.sigma + it.q * n + it.u);
          const uint32_t du = dist_of(a, it.q, it.u);
          for (uint32_t e = it.e0 + ln; e < it.e1; e += 32) push(it, e, su, du);
        },
        a.g);
    if (!grid_barrier(a.ctrl, gen, a.watchdog_ns)) return;
    beg = end;
    count = (uint32_t)*reinterpret_cast<volatile unsigned long long *>(appends);
    ++waves;
  }
  if (gtid == 0) a.cn->waves = waves;
  // largest path count and the 2^53 flag: one atomic per warp
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double y = __shfl_xor_sync(kFull, smax, o);
    smax = y > smax ? y : smax;
  }
  if (lane == 0 && smax > 0.0) {
    atomicMax(&a.cn->sigma_max, (unsigned long long)__double_as_longlong(smax));
    if (smax >= kExactLimit) atomicExch(&a.cn->inexact, 1ull);
  }

  // ---- backward waves: dependencies ------------------------------------------
  for (int32_t t = (int32_t)waves - 1; t >= 0; --t) {
    const uint32_t b = __ldcg(a.wave_off + t), f = __ldcg(a.wave_off + t + 1);
    auto wave_items = [&](int64_t i, int64_t &q, uint32_t &u) {
      const uint2 it = __ldcg(a.wave + b + i);
      q = it.x;
      u = it.y;
    };
    walk_items(
        (int64_t)(f - b), wave_items,
        [&](const Item &it) {
          const double su = __ldcg(a.sigma + it.q * n + it.u);
          const uint32_t du = dist_of(a, it.q, it.u);
          double acc = 0.0;
          for (uint32_t e = it.e0; e < it.e1; ++e) {
            const uint32_t w = __ldg(a.g.adj + e);
            const uint32_t wt = a.weighted ? __ldg(a.g.wt + e) : 1u;
            if (!tight(du, wt, dist_of(a, it.q, w))) continue;
            acc = __dadd_rn(acc, dep_term(su, __ldcg(a.sigma + it.q * n + w), __ldcg(a.delta + it.q * n + w)));
          }
          __stcg(a.delta + it.q * n + it.u, acc);
        },
        [&](const Item &it, int ln) {
          // lanes evaluate 32 arcs at once; the tight terms are then added in
          // arc order (the same additions as one lane walking the arcs)
          const double su = __ldcg(a.sigma + it.q * n + it.u);
          const uint32_t du = dist_of(a, it.q, it.u);
          double acc = 0.0;
          for (uint32_t e0 = it.e0; e0 < it.e1; e0 += 32) {
            const uint32_t e = e0 + ln;
            double term = 0.0;
            bool tt = false;
            if (e < it.e1) {
              const uint32_t w = __ldg(a.g.adj + e);
              const uint32_t wt = a.weighted ? __ldg(a.g.wt + e) : 1u;
              tt = tight(du, wt, dist_of(a, it.q, w));
              if (tt) term = dep_term(su, __ldcg(a.sigma + it.q * n + w), __ldcg(a.delta + it.q * n + w));
            }
            unsigned m = __ballot_sync(kFull, tt);
            while (m) {
              const int j = __ffs(m) - 1;
              m &= m - 1;
              acc = __dadd_rn(acc, __shfl_sync(kFull, term, j));
            }
          }
          if (ln == 0) __stcg(a.delta + it.q * n + it.u, acc);
        },
        a.g);
    if (!grid_barrier(a.ctrl, gen, a.watchdog_ns)) return;
  }

  // ---- gather: bc(v) over the sources in batch order -----------------------------
  for (int64_t u = gtid; u < n; u += nthreads) {
    const int32_t v = a.g.orig ? __ldg(a.g.orig + u) : (int32_t)u;
    double acc = a.accumulate ? a.bc[v] : 0.0;
    for (int32_t q = 0; q < a.nq; ++q)
      if (__ldg(a.src + q) != v) acc = __dadd_rn(acc, __ldcg(a.delta + (int64_t)q * n + u));
    a.bc[v] = acc;
  }
}

// ---- one block per source ---------------------------------------------------
// Road-like graphs (small out-degrees) have deep shortest-path DAGs: the grid
// workload needs about 2,000 waves, each holding only a wavefront of every
// source. There one block runs one source: the waves of a source are
// separated by the block's own barrier instead of a device-wide one, and
// different sources advance independently. The gather over the sources runs
// afterwards as its own launch (bc_gather_kernel). Same operations, same
// order, same results as bc_kernel.
constexpr int kBcBlockThreads = 1024;

__global__ void __launch_bounds__(kBcBlockThreads) bc_block_kernel(BcArgs a) {
  const int64_t n = a.g.n;
  const int64_t q = blockIdx.x;
  const int64_t row = q * n;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  // per-source wave list (n entries) and wave starts (a source has at most n
  // waves, so n + 2 entries), carved from the (query, vertex) buffer read as
  // 32-bit words: it holds 2 * nq * n + 2 * nq of them
  uint32_t *wl = reinterpret_cast<uint32_t *>(a.wave) + row;
  uint32_t *wo = reinterpret_cast<uint32_t *>(a.wave) + (int64_t)a.nq * n + q * (n + 2);
  __shared__ uint32_t s_cnt[3];
  __shared__ int s_bad;
  __shared__ double s_red[kBcBlockThreads / 32];

  for (int64_t i = tid; i < n; i += kBcBlockThreads) {
    a.pc[row + i] = 0u;
    a.sigma[row + i] = 0.0;
    a.delta[row + i] = 0.0;
    if (a.dint) a.dint[row + i] = __ldg(a.dist + row + __ldg(a.g.orig + i));
  }
  const int32_t s = a.src[q];
  if (tid == 0) {
    s_bad = (s < 0 || (int64_t)s >= n || __ldg(a.dist + row + s) != 0u) ? 1 : 0;
    if (s_bad) raise_status(a.ctrl, FG_ERR_INVALID_ARG, kSiteSource);
    s_cnt[0] = s_cnt[1] = s_cnt[2] = 0u;
  }
  __syncthreads();
  if (s_bad) return;
  const uint32_t s_int = a.g.intl ? (uint32_t)a.g.intl[s] : (uint32_t)s;
  if (tid == 0) {
    a.sigma[row + s_int] = 1.0;
    wl[0] = s_int;
    wo[0] = 0u;
    wo[1] = 1u;
  }
  // count tight in-arcs
  for (int64_t u = tid; u < n; u += kBcBlockThreads) {
    const uint32_t du = dist_of(a, q, (uint32_t)u);
    if (du == kInf) continue;
    const uint32_t e0 = __ldg(a.g.rp + u), e1 = __ldg(a.g.rp + u + 1);
    for (uint32_t e = e0; e < e1; ++e) {
      const uint32_t w = __ldg(a.g.adj + e);
      const uint32_t wt = a.weighted ? __ldg(a.g.wt + e) : 1u;
      if (tight(du, wt, dist_of(a, q, w))) atomicAdd(a.pc + row + w, 1u);
    }
  }
  __syncthreads();
  // forward waves; wave t appends through s_cnt[(t + 1) % 3], and the counter
  // of wave t + 1 is cleared during wave t (its last reader passed a barrier)
  double smax = 0.0;
  uint32_t beg = 0, end = 1, waves = 0;
  while (end > beg) {
    if (tid == 0) s_cnt[(waves + 2) % 3] = 0u;
    for (uint32_t i = beg + tid; i < end; i += kBcBlockThreads) {
      const uint32_t u = __ldcg(wl + i);
      const double su = __ldcg(a.sigma + row + u);
      const uint32_t du = dist_of(a, q, u);
      const uint32_t e0 = __ldg(a.g.rp + u), e1 = __ldg(a.g.rp + u + 1);
      for (uint32_t e = e0; e < e1; ++e) {
        const uint32_t w = __ldg(a.g.adj + e);
        const uint32_t wt = a.weighted ? __ldg(a.g.wt + e) : 1u;
        if (!tight(du, wt, dist_of(a, q, w))) continue;
        const double now = atomicAdd(a.sigma + row + w, su) + su;
        smax = now > smax ? now : smax;
        if (atomicSub(a.pc + row + w, 1u) == 1u) {
          const uint32_t pos = end + atomicAdd(&s_cnt[(waves + 1) % 3], 1u);
          if (pos < (uint32_t)n) wl[pos] = w;
          else raise_status(a.ctrl, FG_ERR_INVALID_ARG, kSiteArena);  // cannot happen: each vertex is released once
        }
      }
    }
    __syncthreads();
    const uint32_t added = s_cnt[(waves + 1) % 3];
    beg = end;
    end = end + added;
    ++waves;
    if (tid == 0) wo[waves + 1] = end;
  }
  // largest path count, 2^53 flag, waves: one atomic per block
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double y = __shfl_xor_sync(kFull, smax, o);
    smax = y > smax ? y : smax;
  }
  if (lane == 0) s_red[warp] = smax;
  __syncthreads();
  if (tid == 0) {
    double m = 0.0;
    for (int w = 0; w < kBcBlockThreads / 32; ++w) m = s_red[w] > m ? s_red[w] : m;
    if (m > 0.0) atomicMax(&a.cn->sigma_max, (unsigned long long)__double_as_longlong(m));
    if (m >= kExactLimit) atomicExch(&a.cn->inexact, 1ull);
    atomicMax(&a.cn->waves, (unsigned long long)waves);
  }
  // backward waves: dependencies in CSR order
  for (int32_t t = (int32_t)waves - 1; t >= 0; --t) {
    const uint32_t b = __ldcg(wo + t), f = __ldcg(wo + t + 1);
    for (uint32_t i = b + tid; i < f; i += kBcBlockThreads) {
      const uint32_t u = __ldcg(wl + i);
      const double su = __ldcg(a.sigma + row + u);
      const uint32_t du = dist_of(a, q, u);
      const uint32_t e0 = __ldg(a.g.rp + u), e1 = __ldg(a.g.rp + u + 1);
      double acc = 0.0;
      for (uint32_t e = e0; e < e1; ++e) {
        const uint32_t w = __ldg(a.g.adj + e);
        const uint32_t wt = a.weighted ? __ldg(a.g.wt + e) : 1u;
        if (!tight(du, wt, dist_of(a, q, w))) continue;
        acc = __dadd_rn(acc, dep_term(su, __ldcg(a.sigma + row + w), __ldcg(a.delta + row + w)));
      }
      __stcg(a.delta + row + u, acc);
    }
    __syncthreads();
  }
}

// bc(v) over the sources in batch order (after bc_block_kernel).
__global__ void __launch_bounds__(256) bc_gather_kernel(BcArgs a) {
  const int64_t n = a.g.n;
  for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n; u += (int64_t)gridDim.x * blockDim.x) {
    const int32_t v = a.g.orig ? __ldg(a.g.orig + u) : (int32_t)u;
    double acc = a.accumulate ? a.bc[v] : 0.0;
    for (int32_t q = 0; q < a.nq; ++q)
      if (__ldg(a.src + q) != v) acc = __dadd_rn(acc, __ldcg(a.delta + (int64_t)q * n + u));
    a.bc[v] = acc;
  }
}

}  // namespace
}  // namespace fg

using namespace fg;

extern "C" fg_status fg_bc_accumulate(fg_graph *g, const int32_t *src, int32_t nq, const uint32_t *dist,
                                      int32_t weighted, double *bc, int32_t accumulate, fg_bc_info_t *info,
                                      void *stream_v) {
  if (!g) return fail(FG_ERR_INVALID_ARG, "graph is NULL");
  if (!src || !dist || !bc) return fail(FG_ERR_INVALID_ARG, "src, dist or bc is NULL");
  if (nq <= 0) return fail(FG_ERR_INVALID_ARG, "nq must be > 0 (got %d)", nq);
  if ((reinterpret_cast<uintptr_t>(src) & 3u) || (reinterpret_cast<uintptr_t>(dist) & 3u) ||
      (reinterpret_cast<uintptr_t>(bc) & 7u))
    return fail(FG_ERR_INVALID_ARG, "misaligned pointer");
  if (weighted && !g->weighted) return fail(FG_ERR_INVALID_ARG, "weighted BC on a graph without weights");
  if (weighted && g->has_zero_weight)
    return fail(FG_ERR_UNSUPPORTED, "weighted BC needs positive weights (the graph has an arc of weight 0)");
  const int64_t n = g->n;
  if ((int64_t)nq * n > 0xFFFFFFFFll)
    return fail(FG_ERR_UNSUPPORTED, "nq * n must stay below 2^32 (got %lld); split the batch", (long long)nq * n);
  int dev = -1;
  CUDA_TRY(cudaGetDevice(&dev));
  if (dev != g->device)
    return fail(FG_ERR_INVALID_ARG, "the graph lives on device %d but device %d is current", g->device, dev);
  cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_v);

  std::lock_guard<std::mutex> lk(g->mu);
  BcWorkspace &w = g->bc;
  const size_t cells = (size_t)nq * (size_t)n;
  CUDA_TRY(w.pc.reserve(cells * sizeof(uint32_t)));
  CUDA_TRY(w.sigma.reserve(cells * sizeof(double)));
  CUDA_TRY(w.delta.reserve(cells * sizeof(double)));
  CUDA_TRY(w.wave.reserve(cells * sizeof(uint2) + (size_t)nq * 2 * sizeof(uint32_t)));  // + wave starts (block mode)
  if (g->dg.orig) CUDA_TRY(w.dint.reserve(cells * sizeof(uint32_t)));
  CUDA_TRY(w.wave_off.reserve(((size_t)n + 3) * sizeof(uint32_t)));
  CUDA_TRY(w.ctrl.reserve(sizeof(Ctrl) + sizeof(BcCounters)));
  if (g->bc_blocks == 0) {
    int per_sm = 0, sms = 0;
    CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, bc_kernel, kBcThreads, 0));
    CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    if (per_sm < 1) return fail(FG_ERR_CUDA, "the BC kernel cannot be resident");
    g->bc_blocks = per_sm * sms;
  }
  BcArgs a;
  a.g = g->dg;
  a.nq = nq;
  a.src = src;
  a.dist = dist;
  a.dint = g->dg.orig ? w.dint.as<uint32_t>() : nullptr;
  a.weighted = weighted != 0;
  a.pc = w.pc.as<uint32_t>();
  a.sigma = w.sigma.as<double>();
  a.delta = w.delta.as<double>();
  a.wave = w.wave.as<uint2>();
  a.wave_off = w.wave_off.as<uint32_t>();
  a.bc = bc;
  a.accumulate = accumulate != 0;
  a.ctrl = w.ctrl.as<Ctrl>();
  a.cn = reinterpret_cast<BcCounters *>(w.ctrl.as<unsigned char>() + sizeof(Ctrl));
  a.watchdog_ns = 60ull * 1000000000ull;
  CUDA_TRY(cudaMemsetAsync(a.ctrl, 0, sizeof(Ctrl) + sizeof(BcCounters), stream));
  if (g->max_degree <= kRoadDegree) {
    // road-like: deep DAGs with narrow wavefronts, one block per source
    bc_block_kernel<<<(unsigned)nq, kBcBlockThreads, 0, stream>>>(a);
    CUDA_TRY(cudaGetLastError());
    int sms = 0;
    CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int64_t gblocks = std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, (int64_t)sms * 8));
    bc_gather_kernel<<<(unsigned)gblocks, 256, 0, stream>>>(a);
    CUDA_TRY(cudaGetLastError());
  } else {
    void *args[] = {&a};
    CUDA_TRY(cudaLaunchCooperativeKernel(bc_kernel, dim3(g->bc_blocks), dim3(kBcThreads), args, 0, stream));
  }
  unsigned char hb[sizeof(Ctrl) + sizeof(BcCounters)];
  CUDA_TRY(cudaMemcpyAsync(hb, a.ctrl, sizeof(hb), cudaMemcpyDeviceToHost, stream));
  CUDA_TRY(cudaStreamSynchronize(stream));
  Ctrl h;
  BcCounters hc;
  std::memcpy(&h, hb, sizeof(Ctrl));
  std::memcpy(&hc, hb + sizeof(Ctrl), sizeof(BcCounters));
  if (info) {
    info->waves = (int32_t)hc.waves;
    info->inexact = hc.inexact ? 1 : 0;
    std::memcpy(&info->sigma_max, &hc.sigma_max, sizeof(double));
  }
  switch (h.status) {
    case 0: return FG_OK;
    case FG_ERR_INVALID_ARG:
      return fail(FG_ERR_INVALID_ARG, "a source id is out of range or its distance row does not start at it");
    case FG_ERR_TIMEOUT: return fail(FG_ERR_TIMEOUT, "device barrier timed out");
    default: return fail((fg_status)h.status, "device reported status %d at site %u", h.status, h.site);
  }
}
