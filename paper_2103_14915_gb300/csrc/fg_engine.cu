// Buffered fork-processing engine (Alg. 2) as one persistent cooperative kernel.
//
// One launch runs every round of the buffered loop for a batch of queries:
//
//   INIT      InitBuffers: each query's seed operation <q, src, 0> (PPR: residual 1)
//             goes to the buffer of (partition(src), q)                   (Alg. 2, Sec. 3.2)
//   loop (one round per iteration, device-wide barrier between phases):
//     SCAN-A  per-block totals of buffered operations / non-empty buffers
//     SCAN-B  exclusive scan -> one work item per non-empty (partition, query)
//             buffer ("Consolidate": operations grouped by query, Sec. 4.2,
//             App. B.1 with K = |Q| buckets); ScheduleNextPart (Sec. 5.2):
//             FIFO takes every non-empty buffer, PRIORITY the ones whose best
//             value is within a window of their query's best pending value
//     SCATTER move this round's operations from the append arena into bins
//             ordered by (partition, query)
//     PROCESS IntraPartProcess: each warp claims a work item, stages the
//             query's slice of the partition's state in shared memory, applies
//             the buffered operations, relaxes / pushes inside the partition
//             until done or until a yield heuristic fires (Sec. 5.1), writes the
//             slice back and appends operations for other partitions to the
//             arena (Alg. 2, "send operations to neighbor partitions")
//   until no buffer holds an operation (Alg. 2 loop condition).
//
// A work item is owned by exactly one warp per round, so the query's state
// slice of that partition has a single writer (the atomic-free consolidation
// of Sec. 4.2, here at warp granularity). Operations to other partitions are
// filtered by a plain read of the target's committed value (SSSP/BFS).
#include <cstdio>

#include "fg_device.cuh"

namespace fg {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr uint32_t kMaxVisitSteps = 1u << 22;  // relax/push steps of one visit before the watchdog fires
constexpr uint32_t kBlockChunk = 16;            // work items a block claims at once
constexpr uint32_t kTailChunk = 2;              // ... once fewer than 4 full chunks per block are left
constexpr uint32_t kArenaChunk = 64;            // arena slots a warp reserves at once (>= 32)
constexpr int kLaneMaxDeg = 8;                  // lane-per-vertex expansion for max out-degree <= 8

// Per-warp counters. visits and edges are lane-uniform; spills and yields are
// summed over the lanes when flushed.
struct Counters {
  unsigned long long visits = 0, edges = 0, spills = 0, yields = 0;
};

// Per-warp shared memory: the state slice and five bitmaps of S bits.
struct WarpSmem {
  uint32_t *d;      // [S] distances (u32) or residuals (f32 bits)
  uint32_t *cur;    // [nw] frontier being expanded
  uint32_t *nxt;    // [nw] frontier of the next step
  uint32_t *far;    // [nw] values beyond the current in-visit window
  uint32_t *carry;  // [nw] left for a later visit (yield / spill)
  uint32_t *pfx;    // [nw] exclusive popcount prefix of cur
};

// Per-warp area in words, rounded up to 16 bytes so every warp's slice is
// 16-byte aligned (the dynamic shared memory base is).
__host__ __device__ inline size_t warp_smem_words(int S) {
  return ((size_t)S + 5u * (size_t)(S / 32) + 3u) & ~(size_t)3u;
}


// ---------------------------------------------------------------------------
// Warp-collective append of at most one operation per lane to the arena.
// Per-buffer counts (and best value for priority scheduling) are aggregated
// across lanes that target the same buffer (__match_any_sync). Returns false
// for lanes whose operation did not fit (the caller spills it); lanes without
// an operation return true.
//
// Slots come from the warp's ArenaSlots: the warp reserves kArenaChunk slots
// of the arena at a time, so the device-wide cursor is touched once per chunk
// rather than once per append (a returning atomic on one address that every
// warp of the grid shares). Reserved slots a warp does not fill become holes
// (kInvalidKey) that SCATTER skips. Without ArenaSlots (seeding), each call
// reserves exactly what it appends.
// ---------------------------------------------------------------------------
struct ArenaSlots {
  unsigned long long pos = 0, end = 0;  // lane-uniform: [pos, end) reserved, not yet written
  unsigned long long seen = 0;          // device-wide cursor as of the last reservation
};

// Arena pressure: once a quarter of the arena is left, visits stop at their
// next step and unvisited items are carried to the next round, so a round's
// appends stay within the arena instead of spilling. (A spilled relaxation
// re-marks its source vertex, and re-expanding a vertex of high degree round
// after round multiplies the work.)
__device__ __forceinline__ bool arena_pressed(const EngineArgs &a, unsigned long long cursor) {
  return cursor >= a.e_cap - (a.e_cap >> 2);
}

__device__ __forceinline__ void release_slots(const EngineArgs &a, ArenaSlots &sl) {
  const int lane = lane_id();
  const unsigned long long lim = sl.end < a.e_cap ? sl.end : a.e_cap;
  for (unsigned long long s = sl.pos + (unsigned long long)lane; s < lim; s += 32ull) a.e_key[s] = kInvalidKey;
  sl.pos = sl.end;
}

__device__ __forceinline__ bool emit_ops(const EngineArgs &a, bool has, uint32_t key, uint32_t lv,
                                         uint32_t val, bool track_prio, ArenaSlots *sl = nullptr) {
  const unsigned m = __ballot_sync(kFull, has);
  if (m == 0) return true;
  const int lane = lane_id();
  const unsigned n = (unsigned)__popc(m);
  unsigned long long base = 0;
  if (sl != nullptr) {
    if (sl->pos + n > sl->end) {
      release_slots(a, *sl);
      if (lane == 0) base = atomicAdd(&a.ctrl->e_cursor, (unsigned long long)kArenaChunk);
      base = __shfl_sync(kFull, base, 0);
      sl->pos = base;
      sl->end = base + kArenaChunk;
      sl->seen = sl->end;
    }
    base = sl->pos;
    sl->pos += n;
  } else {
    const int leader = __ffs(m) - 1;
    if (lane == leader) base = atomicAdd(&a.ctrl->e_cursor, (unsigned long long)n);
    base = __shfl_sync(kFull, base, leader);
  }
  const unsigned long long slot = base + (unsigned long long)__popc(m & ((1u << lane) - 1u));
  const bool fits = has && slot < a.e_cap;
  if (fits) {
    a.e_key[slot] = key;
    a.e_op[slot] = make_uint2(lv, val);
  }
  const unsigned fm = __ballot_sync(kFull, fits);
  if (fits) {
    const unsigned grp = __match_any_sync(fm, key);
    const int gl = __ffs(grp) - 1;
    if (track_prio) {
      const uint32_t mn = __reduce_min_sync(grp, val);
      if (lane == gl) atomicMin(&a.prio[key], mn);
    }
    if (lane == gl) atomicAdd(&a.cnt[key], (unsigned)__popc(grp));
  }
  return !has || fits;
}

// Grid-stride fill of count 32-bit words with 16-byte stores for the aligned body.
__device__ __forceinline__ void fill_u32(uint32_t *p, uint64_t count, uint32_t val, uint64_t tid, uint64_t nthr) {
  const uint64_t mis = (reinterpret_cast<uintptr_t>(p) & 15u) >> 2;
  const uint64_t head = mis ? umin64(count, 4u - mis) : 0u;
  if (tid < head) p[tid] = val;
  const uint64_t body = (count - head) / 4u;
  uint4 *q = reinterpret_cast<uint4 *>(p + head);
  const uint4 v4 = make_uint4(val, val, val, val);
  for (uint64_t i = tid; i < body; i += nthr) q[i] = v4;
  const uint64_t tail0 = head + body * 4u;
  if (tid < count - tail0) p[tail0 + tid] = val;
}

// Lane `lane` owns the words [w0, w1) of an nw-word bitmap.
struct WordRange {
  int w0, w1;
  __device__ WordRange(int nw, int lane) {
    const int per = (nw + 31) >> 5;
    w0 = min(nw, lane * per);
    w1 = min(nw, w0 + per);
  }
};

// Build the exclusive popcount prefix of cur; returns the frontier size.
__device__ __forceinline__ uint32_t frontier_prefix(const WarpSmem &w, const WordRange &r) {
  uint32_t tot = 0;
  for (int wd = r.w0; wd < r.w1; ++wd) {
    w.pfx[wd] = tot;
    tot += __popc(w.cur[wd]);
  }
  const uint32_t incl = warp_incl_scan(tot);
  const uint32_t ex = incl - tot;
  for (int wd = r.w0; wd < r.w1; ++wd) w.pfx[wd] += ex;
  __syncwarp();
  return __shfl_sync(kFull, incl, 31);
}

// idx-th set bit of cur (0-based), using the prefix array.
// Register form of the step's frontier, for partitions of at most 1024
// vertices (at most one bitmap word per lane): lane l holds word l of cur,
// the popcount prefix of the words before it, and the total. Selection then
// needs shuffles only (no prefix words in shared memory, no warp sync).
struct RegFrontier {
  uint32_t word, ex, tot;
};

__device__ __forceinline__ RegFrontier reg_frontier(const WarpSmem &w, int nw, int lane) {
  RegFrontier f;
  f.word = lane < nw ? w.cur[lane] : 0u;
  const uint32_t c = (uint32_t)__popc(f.word);
  const uint32_t incl = warp_incl_scan(c);
  f.ex = incl - c;
  f.tot = __shfl_sync(kFull, incl, 31);
  return f;
}

// Position of the r-th set bit (r counted from 0, r < popcount(x)), found by
// halving: compare r with the popcount of the lower half at each width.
__device__ __forceinline__ uint32_t nth_set_bit(uint32_t x, uint32_t r) {
  uint32_t pos = 0;
#pragma unroll
  for (int wd = 16; wd; wd >>= 1) {
    const uint32_t lo = (uint32_t)__popc(x & ((1u << wd) - 1u));
    if (r >= lo) {
      r -= lo;
      x >>= wd;
      pos += (uint32_t)wd;
    }
  }
  return pos;
}

// Vertex (slice index) of frontier position idx < f.tot. Warp-collective:
// every lane calls it (inactive lanes with idx = 0).
__device__ __forceinline__ uint32_t reg_select(const RegFrontier &f, uint32_t idx) {
  const int L = owner_lane(f.ex, idx);  // the lane whose word holds position idx
  const uint32_t wL = __shfl_sync(kFull, f.word, L);
  const uint32_t exL = __shfl_sync(kFull, f.ex, L);
  return (uint32_t)L * 32u + nth_set_bit(wL, idx - exL);
}

__device__ __forceinline__ uint32_t frontier_select(const WarpSmem &w, int nw, uint32_t idx) {
  int lo = 0, hi = nw - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (w.pfx[mid] <= idx) lo = mid; else hi = mid - 1;
  }
  const uint32_t word = w.cur[lo];
  const uint32_t r = idx - w.pfx[lo];
  const int bit = __fns(word, 0, (int)r + 1);
  return (uint32_t)lo * 32u + (uint32_t)bit;
}

// Query state is kept in partition-major (internal) vertex order, so a
// partition's slice of one query is a contiguous run of S values.
__device__ __forceinline__ void load_slice(uint32_t *dst, const uint32_t *src, int Sp, int lane) {
  if (((reinterpret_cast<uintptr_t>(src) | reinterpret_cast<uintptr_t>(dst)) & 15u) == 0 && (Sp & 3) == 0) {
    const uint4 *s4 = reinterpret_cast<const uint4 *>(src);
    uint4 *d4 = reinterpret_cast<uint4 *>(dst);
    for (int i = lane; i < (Sp >> 2); i += 32) d4[i] = __ldcg(s4 + i);
  } else {
    for (int i = lane; i < Sp; i += 32) dst[i] = __ldcg(src + i);
  }
}

__device__ __forceinline__ void store_slice(uint32_t *dst, const uint32_t *src, int Sp, int lane) {
  if (((reinterpret_cast<uintptr_t>(src) | reinterpret_cast<uintptr_t>(dst)) & 15u) == 0 && (Sp & 3) == 0) {
    uint4 *d4 = reinterpret_cast<uint4 *>(dst);
    const uint4 *s4 = reinterpret_cast<const uint4 *>(src);
    for (int i = lane; i < (Sp >> 2); i += 32) __stcg(d4 + i, s4[i]);
  } else {
    for (int i = lane; i < Sp; i += 32) __stcg(dst + i, src[i]);
  }
}

// The resident partition's CSR: prp = rp + partition base, indexed by the
// local vertex id, holding absolute arc offsets into g.adj / g.wt.
// A vertex's arc range must lie inside the arc arrays (never index outside them).
__device__ __forceinline__ bool arcs_in_range(const DevGraph &g, uint32_t e0, uint32_t deg) {
  return (uint64_t)e0 + deg <= g.m;
}

__device__ __forceinline__ uint32_t relax_value(const EngineArgs &a, uint32_t d, uint32_t w) {
  const uint64_t s64 = (uint64_t)d + (uint64_t)w;
  if (s64 >= (uint64_t)kInf) {
    atomicCAS(&a.ctrl->status, 0, (int)FG_ERR_OVERFLOW);
    return kInf - 1u;
  }
  return (uint32_t)s64;
}

// Lower a partition-local vertex and route it: next step (< T), far window
// ([T, Ty)) or a later visit (>= Ty), clearing the bit of its previous class.
__device__ __forceinline__ void relax_local(const WarpSmem &w, uint32_t lu, uint32_t nd, uint32_t T, uint32_t Ty) {
  const uint32_t bit = 1u << (lu & 31);
  const uint32_t old = atomicMin(&w.d[lu], nd);
  if (nd < old) {
    if (nd < T) {
      atomicOr(&w.nxt[lu >> 5], bit);
      if (old != kInf && old >= T) {
        if (old < Ty) atomicAnd(&w.far[lu >> 5], ~bit);
        else atomicAnd(&w.carry[lu >> 5], ~bit);
      }
    } else if (nd < Ty) {
      atomicOr(&w.far[lu >> 5], bit);
      if (old != kInf && old >= Ty) atomicAnd(&w.carry[lu >> 5], ~bit);
    } else {
      atomicOr(&w.carry[lu >> 5], bit);
    }
  }
}

// ---------------------------------------------------------------------------
// SSSP / BFS visit of one (partition, query) buffer.
// ---------------------------------------------------------------------------
template <int QT, bool LANES>
__device__ void visit_dist(const EngineArgs &a, const WarpSmem &w0, uint4 item, uint32_t qbound, const uint32_t *prp,
                           Counters &ctr, ArenaSlots &sl) {
  const DevGraph &g = a.g;
  const int lane = lane_id();
  const uint32_t key = item.x, off = item.y, cnt = item.z, flags = item.w;
  const uint32_t nq = (uint32_t)a.nq;
  const uint32_t p = key / nq, q = key - p * nq;
  const int S = g.S, nw = S >> 5;
  const uint32_t base = p << g.slog2;
  const int Sp = min(S, g.n - (int)base);
  uint32_t *drow = a.dist + (size_t)q * (size_t)g.n;
  WarpSmem w = w0;
  const WordRange wr(nw, lane);

  // 1. stage the query's slice of this partition (bypassing L1)
  load_slice(w.d, drow + base, Sp, lane);
  for (int i = Sp + lane; i < S; i += 32) w.d[i] = kInf;
  for (int wd = lane; wd < nw; wd += 32) {
    w.cur[wd] = 0u; w.nxt[wd] = 0u; w.far[wd] = 0u; w.carry[wd] = 0u;
  }
  // 2. vertices deferred by an earlier visit
  uint32_t *pend = a.pend + (size_t)key * (size_t)nw;
  if (flags & 1u) {
    for (int wd = lane; wd < nw; wd += 32) {
      w.cur[wd] = __ldcg(pend + wd);
      pend[wd] = 0u;
    }
  }
  __syncwarp();
  // 3. apply buffered operations; an operation is live iff it improves the value
  const uint2 *ops = a.b_op + off;
  for (uint32_t j = lane; j < cnt; j += 32) {
    const uint2 o = __ldcg(ops + j);
    const uint32_t old = atomicMin(&w.d[o.x], o.y);
    if (o.y < old) atomicOr(&w.cur[o.x >> 5], 1u << (o.x & 31));
  }
  __syncwarp();
  // 4. in-visit windows: values >= Ty wait for a later visit (yield heuristic 2);
  //    values in [T, Ty) wait for the window to advance (near/far order).
  uint32_t fmin = kInf;
  for (int wd = wr.w0; wd < wr.w1; ++wd) {
    uint32_t b = w.cur[wd];
    while (b) {
      const int t = __ffs(b) - 1;
      b &= b - 1;
      fmin = min(fmin, w.d[wd * 32 + t]);
    }
  }
  fmin = warp_min_u32(fmin);
  if (fmin == kInf) return;  // every operation was stale: the slice is unchanged
  ctr.visits++;
  // values at or beyond Ty stay buffered for a later visit: the yield window
  // (first value + delta) and, under priority scheduling, the query's round
  // bound (best pending value + window), i.e. Delta-stepping across partitions
  const uint32_t Ty = min(a.delta ? sat_add_u32(fmin, a.delta) : kInf, qbound);
  uint32_t T = a.bucket ? min(sat_add_u32(fmin, a.bucket), Ty) : Ty;
  if (T != kInf) {
    for (int wd = wr.w0; wd < wr.w1; ++wd) {
      uint32_t b = w.cur[wd], keep = 0u, fa = 0u, ca = 0u;
      while (b) {
        const int t = __ffs(b) - 1;
        const uint32_t bit = 1u << t;
        b &= b - 1;
        const uint32_t d = w.d[wd * 32 + t];
        if (d < T) keep |= bit; else if (d < Ty) fa |= bit; else ca |= bit;
      }
      w.cur[wd] = keep; w.far[wd] |= fa; w.carry[wd] |= ca;
    }
    __syncwarp();
  }

  uint64_t vis_edges = 0;
  bool stopped = false;
  uint32_t steps = 0;
  for (;;) {
    // bounded loop: a visit can never spin forever
    if (++steps > kMaxVisitSteps || ((steps & 255u) == 0 && ld_volatile_i32(&a.ctrl->abort))) {
      if (steps > kMaxVisitSteps) raise_status(a.ctrl, FG_ERR_TIMEOUT, kSiteVisit);
      stopped = true;
      break;
    }
    uint32_t F;
    RegFrontier rf;
    const bool reg_front = nw <= 32;
    if (LANES) {
      uint32_t cntl = 0;
      for (int wd = wr.w0; wd < wr.w1; ++wd) cntl += __popc(w.cur[wd]);
      F = __reduce_add_sync(kFull, cntl);
    } else if (reg_front) {
      rf = reg_frontier(w, nw, lane);
      F = rf.tot;
    } else {
      F = frontier_prefix(w, wr);
    }
    if (F == 0) {
      // advance the in-visit window to the smallest far value
      uint32_t fm = kInf;
      for (int wd = wr.w0; wd < wr.w1; ++wd) {
        uint32_t b = w.far[wd];
        while (b) {
          const int t = __ffs(b) - 1;
          b &= b - 1;
          fm = min(fm, w.d[wd * 32 + t]);
        }
      }
      fm = warp_min_u32(fm);
      if (fm == kInf) break;
      T = a.bucket ? min(sat_add_u32(fm, a.bucket), Ty) : Ty;
      for (int wd = wr.w0; wd < wr.w1; ++wd) {
        uint32_t b = w.far[wd], mv = 0u;
        while (b) {
          const int t = __ffs(b) - 1;
          b &= b - 1;
          if (w.d[wd * 32 + t] < T) mv |= 1u << t;
        }
        w.far[wd] &= ~mv;
        w.cur[wd] |= mv;
      }
      __syncwarp();
      continue;
    }
    if (a.yield_edges && vis_edges >= a.yield_edges) {  // yield heuristic 1
      stopped = true;
      break;
    }
    if (arena_pressed(a, sl.seen)) {  // leave the rest of the visit to the next round
      stopped = true;
      break;
    }
    if (LANES) {
      // low-degree graphs: each lane expands the frontier vertices of its own
      // bitmap words, loading all arcs of a vertex at once
      const int per = (nw + 31) >> 5;
      for (int k = 0; k < per; ++k) {
        const int wd = wr.w0 + k;
        uint32_t b = (wd < wr.w1) ? w.cur[wd] : 0u;
        while (__any_sync(kFull, b != 0u)) {
          uint32_t v = 0, dv = 0, e0 = 0, deg = 0;
          if (b) {
            const int t = __ffs(b) - 1;
            b &= b - 1;
            v = (uint32_t)wd * 32u + (uint32_t)t;
            dv = w.d[v];
            e0 = prp[v];
            deg = prp[v + 1] - e0;
            if (deg > (uint32_t)kLaneMaxDeg || !arcs_in_range(g, e0, deg)) {  // inconsistent view: skip
              raise_status(a.ctrl, FG_ERR_CUDA, kSiteDegree);
              deg = 0;
            }
          }
          vis_edges += __reduce_add_sync(kFull, deg);
          uint32_t u[kLaneMaxDeg], nd[kLaneMaxDeg];
#pragma unroll
          for (int j = 0; j < kLaneMaxDeg; ++j) {
            u[j] = 0u;
            nd[j] = 0u;
            if ((uint32_t)j < deg) {
              u[j] = g.adj[e0 + j];
              const uint32_t wgt = (QT == Q_BFS || g.wt == nullptr) ? 1u : g.wt[e0 + j];
              nd[j] = relax_value(a, dv, wgt);
            }
          }
          uint32_t extm = 0u;
#pragma unroll
          for (int j = 0; j < kLaneMaxDeg; ++j) {
            if ((uint32_t)j < deg) {
              if ((u[j] >> g.slog2) == p) {
                relax_local(w, u[j] & (uint32_t)(S - 1), nd[j], T, Ty);
              } else if (nd[j] < a.dist[(size_t)q * (size_t)g.n + u[j]]) {
                extm |= 1u << j;
              }
            }
          }
          if (__any_sync(kFull, extm != 0u)) {
#pragma unroll
            for (int j = 0; j < kLaneMaxDeg; ++j) {
              const bool e = (extm >> j) & 1u;
              const uint32_t pk = (u[j] >> g.slog2) * nq + q;
              if (!emit_ops(a, e, pk, u[j] & (uint32_t)(S - 1), nd[j], true, &sl)) {
                atomicOr(&w.carry[v >> 5], 1u << (v & 31));
                ctr.spills++;
              }
            }
          }
        }
      }
      __syncwarp();
    } else {
      // any degree distribution: the batch's arcs are spread evenly over the lanes
      for (uint32_t b0 = 0; b0 < F; b0 += 32) {
        const uint32_t idx = b0 + (uint32_t)lane;
        uint32_t v = 0, dv = 0, a0 = 0, deg = 0;
        if (reg_front) v = reg_select(rf, idx < F ? idx : 0u);
        if (idx < F) {
          if (!reg_front) v = frontier_select(w, nw, idx);
          dv = w.d[v];
          a0 = prp[v];
          deg = prp[v + 1] - a0;
          if (deg > g.max_deg || !arcs_in_range(g, a0, deg)) {  // inconsistent view: skip
            raise_status(a.ctrl, FG_ERR_CUDA, kSiteDegree);
            deg = 0;
          }
        }
        const uint32_t incl = warp_incl_scan(deg);
        const uint32_t exd = incl - deg;
        const uint32_t tot = __shfl_sync(kFull, incl, 31);
        vis_edges += tot;
        for (uint32_t j = 0; j < tot; j += 32) {
          const uint32_t t = j + (uint32_t)lane;
          const bool has = t < tot;
          const int L = owner_lane(exd, has ? t : 0u);
          const uint32_t eL = __shfl_sync(kFull, a0, L) + (t - __shfl_sync(kFull, exd, L));
          const uint32_t du = __shfl_sync(kFull, dv, L);
          const uint32_t vL = __shfl_sync(kFull, v, L);
          uint32_t u = 0, nd = 0;
          bool ext = false;
          if (has) {
            u = g.adj[eL];
            const uint32_t wgt = (QT == Q_BFS || g.wt == nullptr) ? 1u : g.wt[eL];
            nd = relax_value(a, du, wgt);
            if ((u >> g.slog2) == p) {
              relax_local(w, u & (uint32_t)(S - 1), nd, T, Ty);
            } else {
              ext = nd < a.dist[(size_t)q * (size_t)g.n + u];
            }
          }
          const uint32_t pk = (u >> g.slog2) * nq + q;
          if (!emit_ops(a, ext, pk, u & (uint32_t)(S - 1), nd, true, &sl)) {
            atomicOr(&w.carry[vL >> 5], 1u << (vL & 31));
            ctr.spills++;
          }
        }
        __syncwarp();
      }
    }
    // retire the expanded frontier; the next step expands nxt
    for (int wd = wr.w0; wd < wr.w1; ++wd) w.cur[wd] = 0u;
    __syncwarp();
    uint32_t *tmp = w.cur; w.cur = w.nxt; w.nxt = tmp;
  }
  ctr.edges += vis_edges;

  // 5. leftovers -> pending bitmap of this buffer
  uint32_t cmin = kInf;
  bool any = false;
  for (int wd = wr.w0; wd < wr.w1; ++wd) {
    uint32_t b = w.carry[wd];
    if (stopped) b |= w.cur[wd] | w.nxt[wd] | w.far[wd];
    if (b) {
      any = true;
      pend[wd] = b;
      uint32_t bb = b;
      while (bb) {
        const int t = __ffs(bb) - 1;
        bb &= bb - 1;
        cmin = min(cmin, w.d[wd * 32 + t]);
      }
    }
  }
  any = __any_sync(kFull, any);
  cmin = warp_min_u32(cmin);
  if (any && lane == 0) {
    a.dirty[key] = 1u;
    atomicMin(&a.prio[key], cmin);
    ctr.yields++;
  }
  // 6. write the slice back
  __syncwarp();
  store_slice(drow + base, w.d, Sp, lane);
}

// ---------------------------------------------------------------------------
// PPR forward-push visit of one (partition, query) buffer.
// Residuals of the slice live in shared memory; estimates and their Kahan
// compensation are updated in global memory (single writer per slice).
// ---------------------------------------------------------------------------
__device__ __forceinline__ float ppr_thr(const uint32_t *prp, float eps, uint32_t v_local) {
  const uint32_t d = prp[v_local + 1] - prp[v_local];
  return eps * (float)(d > 0u ? d : 1u);
}


__device__ void visit_ppr(const EngineArgs &a, const WarpSmem &w0, uint4 item, const uint32_t *prp, Counters &ctr,
                          ArenaSlots &sl) {
  const DevGraph &g = a.g;
  const int lane = lane_id();
  const uint32_t key = item.x, off = item.y, cnt = item.z, flags = item.w;
  const uint32_t nq = (uint32_t)a.nq;
  const uint32_t p = key / nq, q = key - p * nq;
  const int S = g.S, nw = S >> 5;
  const uint32_t base = p << g.slog2;
  const int Sp = min(S, g.n - (int)base);
  const size_t row = (size_t)q * (size_t)g.n;
  float *rrow = a.pr_r + row;
  float *prow = a.pr_p + row;
  float *crow = a.pr_c + row;
  WarpSmem w = w0;
  float *rs = reinterpret_cast<float *>(w.d);
  const WordRange wr(nw, lane);
  const float alpha = a.alpha, eps = a.eps;
  const float beta = 1.0f - alpha;
  const uint32_t src_int = g.intl ? (uint32_t)g.intl[a.src[q]] : (uint32_t)a.src[q];

  load_slice(w.d, reinterpret_cast<const uint32_t *>(rrow + base), Sp, lane);
  for (int i = Sp + lane; i < S; i += 32) rs[i] = 0.f;
  for (int wd = lane; wd < nw; wd += 32) {
    w.cur[wd] = 0u; w.nxt[wd] = 0u; w.carry[wd] = 0u;
  }
  uint32_t *pend = a.pend + (size_t)key * (size_t)nw;
  if (flags & 1u) {
    for (int wd = lane; wd < nw; wd += 32) {
      w.cur[wd] = __ldcg(pend + wd);
      pend[wd] = 0u;
    }
  }
  __syncwarp();
  const uint2 *ops = a.b_op + off;
  for (uint32_t j = lane; j < cnt; j += 32) {
    const uint2 o = __ldcg(ops + j);
    const float inc = __uint_as_float(o.y);
    const float thr = ppr_thr(prp, eps, o.x);
    const float old = atomicAdd(&rs[o.x], inc);
    if (old < thr && __fadd_rn(old, inc) >= thr) atomicOr(&w.cur[o.x >> 5], 1u << (o.x & 31));
  }
  __syncwarp();

  uint64_t vis_edges = 0;
  bool stopped = false, touched = (cnt > 0) || (flags & 1u);
  uint32_t steps = 0;
  for (;;) {
    if (++steps > kMaxVisitSteps || ((steps & 255u) == 0 && ld_volatile_i32(&a.ctrl->abort))) {
      if (steps > kMaxVisitSteps) raise_status(a.ctrl, FG_ERR_TIMEOUT, kSiteVisit);
      stopped = true;
      break;
    }
    const uint32_t F = frontier_prefix(w, wr);
    if (F == 0) break;
    if (a.yield_edges && vis_edges >= a.yield_edges) {
      stopped = true;
      break;
    }
    for (uint32_t b0 = 0; b0 < F; b0 += 32) {
      const uint32_t idx = b0 + (uint32_t)lane;
      const bool valid = idx < F;
      uint32_t v = 0, a0 = 0, deg = 0;
      if (valid) {
        v = frontier_select(w, nw, idx);
        a0 = prp[v];
        deg = prp[v + 1] - a0;
        if (deg > g.max_deg || !arcs_in_range(g, a0, deg)) {  // inconsistent view: skip
          raise_status(a.ctrl, FG_ERR_CUDA, kSiteDegree);
          deg = 0;
        }
      }
      // arcs this lane's vertex contributes (a dangling vertex sends one
      // operation back to the source)
      const uint32_t arcs = valid ? (deg > 0u ? deg : 1u) : 0u;
      const uint32_t incl = warp_incl_scan(arcs);
      const uint32_t exd = incl - arcs;
      const uint32_t tot = __shfl_sync(kFull, incl, 31);
      // pass 1: count operations for other partitions and reserve them at once
      uint32_t n_ext = 0;
      for (uint32_t j = 0; j < tot; j += 32) {
        const uint32_t t = j + (uint32_t)lane;
        const bool has = t < tot;
        const int L = owner_lane(exd, has ? t : 0u);
        const uint32_t degL = __shfl_sync(kFull, deg, L);
        const uint32_t eL = __shfl_sync(kFull, a0, L) + (t - __shfl_sync(kFull, exd, L));
        bool ext = false;
        if (has) {
          const uint32_t u = degL > 0u ? g.adj[eL] : src_int;
          ext = (u >> g.slog2) != p;
        }
        n_ext += __popc(__ballot_sync(kFull, ext));
      }
      // reserve the batch's cross-partition increments together, from the
      // warp's own arena chunk (a new chunk of at least kArenaChunk slots
      // when it runs short)
      unsigned long long rbase = 0;
      if (n_ext) {
        if (sl.pos + n_ext > sl.end) {
          release_slots(a, sl);
          const unsigned long long want = n_ext > kArenaChunk ? (unsigned long long)n_ext : kArenaChunk;
          unsigned long long b = 0;
          if (lane == 0) b = atomicAdd(&a.ctrl->e_cursor, want);
          b = __shfl_sync(kFull, b, 0);
          sl.pos = b;
          sl.end = b + want;
          sl.seen = sl.end;
        }
        rbase = sl.pos;
        sl.pos += n_ext;
      }
      if (n_ext && rbase + n_ext > a.e_cap) {
        // does not fit this round: keep these vertices for a later visit
        if (n_ext > a.e_cap) raise_status(a.ctrl, FG_ERR_BIN_OVERFLOW, kSiteArena);
        for (unsigned long long s = rbase + lane; s < a.e_cap && s < rbase + n_ext; s += 32)
          a.e_key[s] = kInvalidKey;
        if (valid) atomicOr(&w.carry[v >> 5], 1u << (v & 31));
        if (lane == 0) ctr.spills++;
        __syncwarp();
        continue;
      }
      // take the residuals and move alpha * rho into the estimates (Kahan)
      float rho = 0.f, inc_l = 0.f;
      if (valid) {
        rho = atomicExch(&rs[v], 0.f);
        const uint32_t gi = base + v;
        const float pe = __ldcg(prow + gi), ce = __ldcg(crow + gi);
        const float y = __fsub_rn(__fmul_rn(alpha, rho), ce);
        const float tsum = __fadd_rn(pe, y);
        __stcg(crow + gi, __fsub_rn(__fsub_rn(tsum, pe), y));
        __stcg(prow + gi, tsum);
        inc_l = deg > 0u ? __fdiv_rn(__fmul_rn(beta, rho), (float)deg) : __fmul_rn(beta, rho);
      }
      vis_edges += tot;
      // pass 2: spread (1 - alpha) rho
      uint32_t run = 0;
      for (uint32_t j = 0; j < tot; j += 32) {
        const uint32_t t = j + (uint32_t)lane;
        const bool has = t < tot;
        const int L = owner_lane(exd, has ? t : 0u);
        const uint32_t degL = __shfl_sync(kFull, deg, L);
        const uint32_t eL = __shfl_sync(kFull, a0, L) + (t - __shfl_sync(kFull, exd, L));
        const float inc = __shfl_sync(kFull, inc_l, L);
        bool ext = false;
        uint32_t u = 0;
        if (has) {
          u = degL > 0u ? g.adj[eL] : src_int;
          if ((u >> g.slog2) == p) {
            const uint32_t lu = u & (uint32_t)(S - 1);
            const float thr = ppr_thr(prp, eps, lu);
            const float old = atomicAdd(&rs[lu], inc);
            if (old < thr && __fadd_rn(old, inc) >= thr) atomicOr(&w.nxt[lu >> 5], 1u << (lu & 31));
          } else {
            ext = true;
          }
        }
        const unsigned em = __ballot_sync(kFull, ext);
        if (ext) {
          const unsigned long long slot = rbase + run + __popc(em & ((1u << lane) - 1u));
          const uint32_t pk = (u >> g.slog2) * nq + q;
          a.e_key[slot] = pk;
          a.e_op[slot] = make_uint2(u & (uint32_t)(S - 1), __float_as_uint(inc));
          const unsigned grp = __match_any_sync(em, pk);
          if (lane == __ffs(grp) - 1) atomicAdd(&a.cnt[pk], (unsigned)__popc(grp));
        }
        run += __popc(em);
      }
      __syncwarp();
    }
    for (int wd = wr.w0; wd < wr.w1; ++wd) w.cur[wd] = 0u;
    __syncwarp();
    uint32_t *tmp = w.cur; w.cur = w.nxt; w.nxt = tmp;
  }
  ctr.edges += vis_edges;
  if (touched) ctr.visits++;

  bool any = false;
  for (int wd = wr.w0; wd < wr.w1; ++wd) {
    uint32_t b = w.carry[wd];
    if (stopped) b |= w.cur[wd] | w.nxt[wd];
    if (b) {
      any = true;
      pend[wd] = b;
    }
  }
  any = __any_sync(kFull, any);
  if (any && lane == 0) {
    a.dirty[key] = 1u;
    ctr.yields++;
  }
  __syncwarp();
  store_slice(reinterpret_cast<uint32_t *>(rrow + base), w.d, Sp, lane);
}

// Coin of the random scheduler: a 32-bit mix of (key, round) (the finalizer
// of MurmurHash3, Appleby 2011).
__device__ __forceinline__ uint32_t sched_coin(uint32_t key, uint32_t round) {
  uint32_t x = key * 0x9E3779B1u ^ (round + 1u) * 0x85EBCA77u;
  x ^= x >> 16;
  x *= 0x85EBCA6Bu;
  x ^= x >> 13;
  x *= 0xC2B2AE35u;
  x ^= x >> 16;
  return x;
}

// Buffer skipped by priority scheduling this round (SSSP/BFS). No warp stages
// this (partition, query) slice in the current round, so its operations are
// applied directly to the query's state with atomicMin and the improved
// vertices join the buffer's pending bitmap; the buffer stays non-empty.
__device__ void carry_item(const EngineArgs &a, uint4 item, uint32_t item_prio) {
  const DevGraph &g = a.g;
  const int lane = lane_id();
  const uint32_t key = item.x, off = item.y, cnt = item.z;
  const uint32_t nq = (uint32_t)a.nq;
  const uint32_t p = key / nq, q = key - p * nq;
  const uint32_t base = p << g.slog2;
  const int nw = g.S >> 5;
  uint32_t *drow = a.dist + (size_t)q * (size_t)g.n;
  uint32_t *pend = a.pend + (size_t)key * (size_t)nw;
  bool any = false;
  for (uint32_t j = lane; j < cnt; j += 32) {
    const uint2 o = __ldcg(a.b_op + off + j);
    const uint32_t old = atomicMin(drow + base + o.x, o.y);
    if (o.y < old) {
      atomicOr(pend + (o.x >> 5), 1u << (o.x & 31));
      any = true;
    }
  }
  any = __any_sync(kFull, any) || (item.w & 1u);
  if (any && lane == 0) {
    a.dirty[key] = 1u;
    atomicMin(&a.prio[key], item_prio);
  }
}

// ---------------------------------------------------------------------------
// Block-wide exclusive scan of one u64 per thread.
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long block_excl_scan(unsigned long long x, unsigned long long *s_warp,
                                                              unsigned long long &total) {
  const int lane = lane_id(), wid = threadIdx.x >> 5;
  const unsigned long long incl = warp_incl_scan(x);
  if (lane == 31) s_warp[wid] = incl;
  block_sync();
  if (wid == 0) {
    unsigned long long v = lane < kWarps ? s_warp[lane] : 0ull;
    const unsigned long long vi = warp_incl_scan(v);
    if (lane < kWarps) s_warp[lane] = vi - v;
    if (lane == kWarps - 1) s_warp[kWarps] = vi;
  }
  block_sync();
  const unsigned long long ex = s_warp[wid] + incl - x;
  total = s_warp[kWarps];
  block_sync();
  return ex;
}

// Block-level work claiming. *claim packs (end << 32 | next) for the block's
// current chunk of item indices; the one warp that draws next == end refills
// the chunk from the device-wide counter, warps that draw past the end wait
// for the refill. Chunks are consecutive items (ordered by partition, then
// query), so the warps of one block mostly visit the same partition and read
// its CSR through the SM's L1. Called by one lane; returns an index >= tot
// when the round has no work left for this block.
__device__ uint32_t claim_item(Ctrl *c, unsigned long long *claim, volatile int *done, uint32_t tot,
                               uint64_t watchdog_ns) {
  uint64_t t0 = 0;
  unsigned spins = 0;
  for (;;) {
    if (*done) return kInvalidKey;
    const unsigned long long old = atomicAdd(claim, 1ull);
    const uint32_t pos = (uint32_t)old, end = (uint32_t)(old >> 32);
    if (pos < end) return pos;
    if (pos == end) {
      // full chunks while plenty of work is left; near the end of the round
      // small ones, so that no block takes several visits per warp into the tail
      const uint32_t seen = *reinterpret_cast<volatile uint32_t *>(&c->item_next);
      const uint32_t left = seen < tot ? tot - seen : 0u;
      const uint32_t chunk = left > 4u * kBlockChunk * gridDim.x ? kBlockChunk : kTailChunk;
      uint32_t b = atomicAdd(&c->item_next, chunk);
      if (ld_volatile_i32(&c->abort)) b = tot;
      if (b >= tot) {
        *done = 1;
        return kInvalidKey;
      }
      const uint32_t e = min(tot, b + chunk);
      atomicExch(claim, ((unsigned long long)e << 32) | (unsigned long long)(b + 1u));
      return b;
    }
    // another warp is refilling: wait until the chunk end moves (bounded)
    while ((uint32_t)(*reinterpret_cast<volatile unsigned long long *>(claim) >> 32) == end && !*done) {
      if ((++spins & 63u) == 0) {
        const uint64_t t = global_ns();
        if (t0 == 0) t0 = t;
        else if (t - t0 > watchdog_ns) {
          raise_status(c, FG_ERR_TIMEOUT, kSiteClaim);
          *done = 1;
          return kInvalidKey;
        }
      }
      __nanosleep(32);
    }
  }
}

template <int QT>
__global__ void __launch_bounds__(kThreads, 3) engine_kernel(EngineArgs a) {
  extern __shared__ __align__(16) uint32_t smem_dyn[];
  __shared__ unsigned long long s_scan[kWarps + 1];
  __shared__ unsigned long long s_pre[4];
  __shared__ unsigned long long s_hv[kWarps];
  __shared__ unsigned long long s_claim;  // block's chunk of work items (claim_item)
  __shared__ int s_claim_done;
  constexpr bool kPPR = (QT == Q_PPR);

  const int lane = lane_id(), wid = threadIdx.x >> 5;
  const int S = a.g.S, nw = S >> 5;
  WarpSmem w;
  {
    uint32_t *b = smem_dyn + (size_t)wid * warp_smem_words(S);
    w.d = b;
    w.cur = b + S;
    w.nxt = w.cur + nw;
    w.far = w.nxt + nw;
    w.carry = w.far + nw;
    w.pfx = w.carry + nw;
  }
  Ctrl *c = a.ctrl;
  // every block reads the generation before its first arrival, so all agree
  unsigned gen = *reinterpret_cast<volatile unsigned *>(&c->bar_gen);
  Counters ctr;
  // phase clock of block 0 (device time between device-wide barriers)
  uint64_t t_prev = (blockIdx.x == 0 && threadIdx.x == 0) ? global_ns() : 0ull;
  unsigned long long ph[6] = {0ull, 0ull, 0ull, 0ull, 0ull, 0ull};
#define FG_PHASE(k)                                             \
  do {                                                          \
    if (blockIdx.x == 0 && threadIdx.x == 0) {                  \
      const uint64_t t_now = global_ns();                       \
      ph[k] += t_now - t_prev;                                  \
      t_prev = t_now;                                           \
    }                                                           \
  } while (0)
  const uint64_t K = (uint64_t)a.g.nparts * (uint64_t)a.nq;
  const uint64_t per_blk = (K + gridDim.x - 1) / gridDim.x;
  const uint64_t k0 = umin64(K, (uint64_t)blockIdx.x * per_blk);
  const uint64_t k1 = umin64(K, k0 + per_blk);
  const uint32_t gwarp = blockIdx.x * kWarps + wid, nwarps = gridDim.x * kWarps;

  // ---- K0: state tiles and per-buffer counters (InitBuffers, first half) ----
  {
    const uint64_t rows = (uint64_t)a.nq * (uint64_t)a.g.n;
    const uint64_t tid = (uint64_t)blockIdx.x * kThreads + threadIdx.x, nthr = (uint64_t)gridDim.x * kThreads;
    if (kPPR) {
      fill_u32(reinterpret_cast<uint32_t *>(a.pr_p), rows, 0u, tid, nthr);
      fill_u32(reinterpret_cast<uint32_t *>(a.pr_r), rows, 0u, tid, nthr);
      fill_u32(reinterpret_cast<uint32_t *>(a.pr_c), rows, 0u, tid, nthr);
    } else {
      fill_u32(a.dist, rows, kInf, tid, nthr);
      fill_u32(a.prio, K, kInf, tid, nthr);
      fill_u32(a.qbest, 2u * (uint64_t)a.nq, kInf, tid, nthr);
    }
    fill_u32(a.cnt, K, 0u, tid, nthr);
    fill_u32(a.dirty, K, 0u, tid, nthr);
  }
  if (!grid_barrier(c, gen, a.watchdog_ns)) goto done;
  FG_PHASE(0);

  // ---- INIT: seed operations (InitBuffers, second half) ----
  for (uint32_t q0 = gwarp * 32u; q0 < (uint32_t)a.nq; q0 += nwarps * 32u) {
    const uint32_t q = q0 + lane;
    bool has = q < (uint32_t)a.nq;
    uint32_t key = 0, lv = 0;
    if (has && (a.src[q] < 0 || a.src[q] >= a.g.n)) {
      raise_status(c, FG_ERR_INVALID_ARG, kSiteSource);  // source id out of range
      has = false;
    }
    if (has) {
      const int32_t s = a.src[q];
      const uint32_t v = a.g.intl ? (uint32_t)a.g.intl[s] : (uint32_t)s;
      key = (v >> a.g.slog2) * (uint32_t)a.nq + q;
      lv = v & (uint32_t)(S - 1);
    }
    const uint32_t val0 = kPPR ? __float_as_uint(1.0f) : 0u;
    const bool ok = emit_ops(a, has, key, lv, val0, !kPPR);
    if (!ok) raise_status(c, FG_ERR_BIN_OVERFLOW, kSiteArena);
  }
  if (!grid_barrier(c, gen, a.watchdog_ns)) goto done;
  FG_PHASE(1);

  for (uint32_t round = 0;; ++round) {
    // best pending value per query: written in SCAN-A, read in SCAN-B and PROCESS,
    // and the other half is cleared in SCATTER for the next round
    uint32_t *qb_cur = a.qbest + (size_t)(round & 1u) * (size_t)a.nq;
    uint32_t *qb_nxt = a.qbest + (size_t)((round + 1u) & 1u) * (size_t)a.nq;
    // ---- SCAN-A: per-block totals ----
    {
      unsigned long long loc = 0, hv = 0;
      uint32_t mx = 0;  // largest buffer of the round (max-operations scheduling)
#pragma unroll 4
      for (uint64_t k = k0 + threadIdx.x; k < k1; k += kThreads) {
        const uint32_t n_ops = __ldcg(a.cnt + k);
        const bool dk = __ldcg(a.dirty + k) != 0u;
        const bool act = n_ops > 0u || dk;
        loc += ((unsigned long long)n_ops << 32) | (act ? 1ull : 0ull);
        hv += dk ? 1ull : 0ull;
        if (!kPPR && act && a.sched == FG_SCHED_PRIORITY)
          atomicMin(&qb_cur[(uint32_t)k % (uint32_t)a.nq], __ldcg(a.prio + k));
        if (!kPPR && a.sched == FG_SCHED_MAXOPS) mx = n_ops > mx ? n_ops : mx;
      }
      if (!kPPR && a.sched == FG_SCHED_MAXOPS) {
        mx = __reduce_max_sync(kFull, mx);
        if (lane == 0 && mx > 0u) atomicMax(&c->max_ops[round & 1u], mx);
      }
      loc = warp_sum(loc);
      hv = warp_sum(hv);
      if (lane == 0) { s_scan[wid] = loc; s_hv[wid] = hv; }
      block_sync();
      if (threadIdx.x == 0) {
        unsigned long long t = 0, th = 0;
        for (int i = 0; i < kWarps; ++i) { t += s_scan[i]; th += s_hv[i]; }
        a.blocksum[blockIdx.x] = t;
        a.blocksum[gridDim.x + blockIdx.x] = th;
      }
    }
    if (!grid_barrier(c, gen, a.watchdog_ns)) goto done;
    FG_PHASE(2);
    // ---- SCAN-B: work items, bin offsets, buffer reset ----
    unsigned long long tot_ops, tot_items, emitted;
    {
      unsigned long long pre = 0, all = 0, preh = 0, allh = 0;
      for (int i = threadIdx.x; i < (int)gridDim.x; i += kThreads) {
        const unsigned long long v = __ldcg(a.blocksum + i);
        const unsigned long long vh = __ldcg(a.blocksum + gridDim.x + i);
        all += v;
        allh += vh;
        if (i < (int)blockIdx.x) { pre += v; preh += vh; }
      }
      pre = warp_sum(pre);
      all = warp_sum(all);
      preh = warp_sum(preh);
      allh = warp_sum(allh);
      if (lane == 0) { s_hv[wid] = preh; }
      block_sync();
      if (threadIdx.x == 0) {
        unsigned long long t = 0;
        for (int i = 0; i < kWarps; ++i) t += s_hv[i];
        s_pre[2] = t;
      }
      block_sync();
      if (lane == 0) { s_hv[wid] = allh; }
      block_sync();
      if (threadIdx.x == 0) {
        unsigned long long t = 0;
        for (int i = 0; i < kWarps; ++i) t += s_hv[i];
        s_pre[3] = t;
      }
      block_sync();
      if (lane == 0) s_scan[wid] = pre;
      block_sync();
      if (threadIdx.x == 0) {
        unsigned long long t = 0;
        for (int i = 0; i < kWarps; ++i) t += s_scan[i];
        s_pre[0] = t;
      }
      block_sync();
      if (lane == 0) s_scan[wid] = all;
      block_sync();
      if (threadIdx.x == 0) {
        unsigned long long t = 0;
        for (int i = 0; i < kWarps; ++i) t += s_scan[i];
        s_pre[1] = t;
      }
      block_sync();
      pre = s_pre[0];
      all = s_pre[1];
      tot_ops = all >> 32;
      tot_items = all & 0xFFFFFFFFull;
      emitted = umin64(*reinterpret_cast<volatile unsigned long long *>(&c->e_cursor), a.e_cap);
      block_sync();
      if (tot_items == 0) break;
      if (round >= a.max_rounds) {
        if (threadIdx.x == 0) raise_status(c, FG_ERR_TIMEOUT, kSiteRounds);
        break;
      }
      unsigned long long run_ops = pre >> 32, run_items = pre & 0xFFFFFFFFull, run_h = s_pre[2];
      const unsigned long long H = s_pre[3];
      const uint32_t window = a.sched_window;
      // tiles of kThreads keys; the next tile's counters are loaded while the
      // current one is scanned and written (the block scan synchronises)
      const bool by_window = !kPPR && a.sched == FG_SCHED_PRIORITY;
      const uint32_t round_max = (!kPPR && a.sched == FG_SCHED_MAXOPS)
                                     ? *reinterpret_cast<volatile unsigned *>(&c->max_ops[round & 1u])
                                     : 0u;
      uint32_t nx_ops = 0, nx_dirty = 0, nx_prio = kInf, nx_qb = kInf;
      {
        const uint64_t k = k0 + threadIdx.x;
        if (k < k1) {
          nx_ops = __ldcg(a.cnt + k);
          nx_dirty = __ldcg(a.dirty + k);
          if (!kPPR) nx_prio = __ldcg(a.prio + k);
          if (by_window) nx_qb = __ldcg(qb_cur + (uint32_t)k % (uint32_t)a.nq);
        }
      }
      for (uint64_t t0 = k0; t0 < k1; t0 += kThreads) {
        const uint64_t k = t0 + threadIdx.x;
        const uint32_t n_ops = nx_ops, dflag = nx_dirty, pr = nx_prio, qb = nx_qb;
        const bool act = k < k1 && (n_ops > 0u || dflag != 0u);
        {
          const uint64_t kn = k + kThreads;
          nx_ops = 0u;
          nx_dirty = 0u;
          nx_prio = kInf;
          nx_qb = kInf;
          if (kn < k1) {
            nx_ops = __ldcg(a.cnt + kn);
            nx_dirty = __ldcg(a.dirty + kn);
            if (!kPPR) nx_prio = __ldcg(a.prio + kn);
            if (by_window) nx_qb = __ldcg(qb_cur + (uint32_t)kn % (uint32_t)a.nq);
          }
        }
        const bool heavy = act && dflag != 0u;
        const unsigned long long x = ((unsigned long long)n_ops << 32) | (act ? 1ull : 0ull) | (heavy ? (1ull << 16) : 0ull);
        unsigned long long tile_tot;
        const unsigned long long ex = block_excl_scan(x, s_scan, tile_tot);
        if (act) {
          const unsigned long long I = run_items + (ex & 0xFFFFull), J = run_h + ((ex >> 16) & 0xFFFFull);
          const uint32_t item_idx = (uint32_t)(heavy ? J : H + I - J);
          const uint32_t off = (uint32_t)(run_ops + (ex >> 32));
          uint32_t fl = dflag ? 1u : 0u;
          if (!kPPR) {
            if (by_window && pr > sat_add_u32(qb, window)) fl |= 2u;
            // Max-#ops and Random (Tab. 4A) in round form: a buffer without
            // carried-over work waits one round when it holds under a quarter
            // of the round's largest buffer, or when a coin drawn from (key,
            // round) says so; it then carries its work and is taken next round
            if (dflag == 0u && a.sched == FG_SCHED_MAXOPS && 4ull * (unsigned long long)n_ops < round_max)
              fl |= 2u;
            if (dflag == 0u && a.sched == FG_SCHED_RANDOM && (sched_coin((uint32_t)k, round) & 1u)) fl |= 2u;
            a.prio[k] = kInf;
          }
          a.items[item_idx] = make_uint4((uint32_t)k, off, n_ops, fl);
          if (!kPPR) a.iprio[item_idx] = pr;
          a.cur[k] = off;
          a.cnt[k] = 0u;
          a.dirty[k] = 0u;
        }
        run_ops += tile_tot >> 32;
        run_items += tile_tot & 0xFFFFull;
        run_h += (tile_tot >> 16) & 0xFFFFull;
      }
      if (blockIdx.x == 0 && threadIdx.x == 0) {
        c->rounds += 1ull;
        c->ops += tot_ops;
        if (tot_ops > c->max_round_ops) c->max_round_ops = tot_ops;
      }
    }
    if (!grid_barrier(c, gen, a.watchdog_ns)) goto done;
    FG_PHASE(3);
    // ---- SCATTER: arena -> bins ordered by (partition, query) ----
    {
      if (blockIdx.x == 0 && threadIdx.x == 0) {
        c->e_cursor = 0ull;
        c->item_next = 0u;
        c->max_ops[(round + 1u) & 1u] = 0u;
      }
      if (threadIdx.x == 0) {  // visible to the block after the barrier below
        s_claim = 0ull;
        s_claim_done = 0;
      }
      if (!kPPR && a.sched == FG_SCHED_PRIORITY)
        for (uint32_t i = blockIdx.x * kThreads + threadIdx.x; i < (uint32_t)a.nq; i += gridDim.x * kThreads)
          qb_nxt[i] = kInf;
      const unsigned long long n_emit = emitted;
      for (unsigned long long i0 = (unsigned long long)gwarp * 32ull; i0 < n_emit; i0 += (unsigned long long)nwarps * 32ull) {
        const unsigned long long i = i0 + lane;
        const bool has0 = i < n_emit;
        uint32_t key = kInvalidKey;
        uint2 o = make_uint2(0u, 0u);
        if (has0) {
          key = __ldcg(a.e_key + i);
          o = __ldcg(a.e_op + i);
        }
        const bool has = has0 && key != kInvalidKey;
        const unsigned m = __ballot_sync(kFull, has);
        if (has) {
          const unsigned grp = __match_any_sync(m, key);
          const int gl = __ffs(grp) - 1;
          uint32_t pos = 0;
          if (lane == gl) pos = atomicAdd(&a.cur[key], (unsigned)__popc(grp));
          pos = __shfl_sync(grp, pos, gl) + __popc(grp & ((1u << lane) - 1u));
          a.b_op[pos] = o;
        }
      }
      (void)tot_ops;
    }
    if (!grid_barrier(c, gen, a.watchdog_ns)) goto done;
    FG_PHASE(4);
    // ---- PROCESS: IntraPartProcess of every work item ----
    // Items are handed out by claim_item (block-level chunks). The resident
    // partition lives in L1/L2: the graph and the round's active state slices
    // fit in L2. No block-level synchronisation here.
    {
      ArenaSlots sl;
      for (;;) {
        uint32_t idx = 0;
        if (lane == 0) idx = claim_item(c, &s_claim, &s_claim_done, (uint32_t)tot_items, a.watchdog_ns);
        idx = __shfl_sync(kFull, idx, 0);
        if (idx >= (uint32_t)tot_items) break;
        const uint4 it = __ldcg(a.items + idx);
        const uint32_t p = it.x / (uint32_t)a.nq;
        const uint32_t *prp = a.g.rp + ((size_t)p << a.g.slog2);
        bool defer = !kPPR && (it.w & 2u);
        if (!kPPR && !defer) {
          unsigned long long cursor = 0;
          if (lane == 0) cursor = *reinterpret_cast<volatile unsigned long long *>(&c->e_cursor);
          cursor = __shfl_sync(kFull, cursor, 0);
          defer = arena_pressed(a, cursor > sl.seen ? cursor : sl.seen);
        }
        if (defer) {
          carry_item(a, it, __ldcg(a.iprio + idx));
        } else if (kPPR) {
          visit_ppr(a, w, it, prp, ctr, sl);
        } else {
          const uint32_t q = it.x - p * (uint32_t)a.nq;
          const uint32_t qbound =
              a.sched == FG_SCHED_PRIORITY ? sat_add_u32(__ldcg(qb_cur + q), a.sched_window) : kInf;
          if (a.lanes) visit_dist<QT, true>(a, w, it, qbound, prp, ctr, sl);
          else visit_dist<QT, false>(a, w, it, qbound, prp, ctr, sl);
        }
      }
      release_slots(a, sl);  // before the barrier: SCATTER reads every reserved slot
    }
    if (!grid_barrier(c, gen, a.watchdog_ns)) goto done;
    FG_PHASE(5);
  }
done:
#undef FG_PHASE
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    const uint64_t t_now = global_ns();
    ph[3] += t_now - t_prev;  // the final scan that found no work
    for (int k = 0; k < 6; ++k) atomicAdd(&c->phase_ns[k], ph[k]);
  }
  {
    const unsigned long long sp = warp_sum(ctr.spills), yl = warp_sum(ctr.yields);
    if (lane == 0) {
      atomicAdd(&c->visits, ctr.visits);
      atomicAdd(&c->edges, ctr.edges);
      atomicAdd(&c->arcs_read, ctr.edges);
      atomicAdd(&c->spills, sp);
      atomicAdd(&c->yields, yl);
    }
  }
}

// ---------------------------------------------------------------------------
// Per-query mass check (PPR): fold the Kahan compensation into the estimate
// (p_out = p - c, FP32) and accumulate sum(p_out) + sum(r) in FP64.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) ppr_finalize_kernel(const float *p, const float *cmp, const float *r,
                                                           float *p_out, float *r_out, const int32_t *orig, int64_t n,
                                                           int64_t chunks, double *mass) {
  __shared__ double s_red[8];
  const int64_t q = blockIdx.x / chunks, ch = blockIdx.x % chunks;
  const int64_t per = (n + chunks - 1) / chunks;
  const int64_t i0 = ch * per, i1 = i0 + per < n ? i0 + per : n;
  const float *prow = p + q * n;
  const float *crow = cmp + q * n;
  const float *rrow = r + q * n;
  float *porow = p_out + q * n;
  float *rorow = r_out ? r_out + q * n : nullptr;
  double acc = 0.0;
  for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
    const float pf = __fsub_rn(prow[i], crow[i]);
    const float rf = rrow[i];
    const int64_t o = orig ? (int64_t)orig[i] : i;
    porow[o] = pf;
    if (rorow && rorow != rrow) rorow[o] = rf;
    acc += (double)pf + (double)rf;
  }
  if (mass) {
    acc = warp_sum(acc);
    if (lane_id() == 0) s_red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += s_red[i];
      atomicAdd(mass + q, t);
    }
  }
}

// Query-major state in internal order -> caller's output in original order.
__global__ void __launch_bounds__(256) permute_out_kernel(const uint32_t *state, uint32_t *out, const int32_t *orig,
                                                          int64_t n, int64_t rows) {
  const int64_t total = n * rows;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t q = t / n, i = t - q * n;
    out[q * n + orig[i]] = state[t];
  }
}

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
static const void *engine_fn(int qtype) {
  switch (qtype) {
    case Q_SSSP: return (const void *)engine_kernel<Q_SSSP>;
    case Q_BFS: return (const void *)engine_kernel<Q_BFS>;
    default: return (const void *)engine_kernel<Q_PPR>;
  }
}

cudaError_t engine_grid_size(int qtype, int S, int *blocks, int *threads, size_t *smem) {
  const void *fn = engine_fn(qtype);
  *threads = kThreads;
  *smem = (size_t)kWarps * warp_smem_words(S) * sizeof(uint32_t);
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)*smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0, dev = 0, sms = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kThreads, *smem);
  if (e != cudaSuccess) return e;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  *blocks = per_sm * sms;
  return cudaSuccess;
}

cudaError_t launch_engine(const EngineArgs &a, int blocks, int threads, size_t smem, cudaStream_t s) {
  EngineArgs copy = a;
  void *args[] = {(void *)&copy};
  return cudaLaunchCooperativeKernel(engine_fn(a.qtype), dim3(blocks), dim3(threads), args, smem, s);
}

cudaError_t launch_ppr_finalize(const EngineArgs &a, double *mass, float *p_out, float *r_out, cudaStream_t s) {
  const int64_t n = a.g.n;
  const int64_t chunks = (n + 4095) / 4096;
  const int64_t grid = chunks * (int64_t)a.nq;
  if (grid <= 0) return cudaSuccess;
  ppr_finalize_kernel<<<(unsigned)grid, 256, 0, s>>>(a.pr_p, a.pr_c, a.pr_r, p_out, r_out, a.g.orig, n, chunks, mass);
  return cudaGetLastError();
}

cudaError_t launch_permute_out(const uint32_t *state, uint32_t *out, const int32_t *orig, int64_t n, int64_t rows,
                               cudaStream_t s) {
  const int64_t total = n * rows;
  if (total <= 0) return cudaSuccess;
  int dev = 0, sms = 0;
  cudaError_t e;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  const int64_t want = (total + 255) / 256;
  const unsigned grid = (unsigned)(want < (int64_t)sms * 16 ? want : (int64_t)sms * 16);
  permute_out_kernel<<<grid, 256, 0, s>>>(state, out, orig, n, rows);
  return cudaGetLastError();
}

}  // namespace fg
