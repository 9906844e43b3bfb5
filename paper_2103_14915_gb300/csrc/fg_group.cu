// Group engine: the buffered loop of Alg. 2 for SSSP and BFS with queries
// processed in groups of G (8, 16 or 32), one lane per query.
//
// Why groups. On graphs whose partitions are cut by almost every arc (power-law
// graphs with the paper's random equal-vertex partitions, Sec. 6.1), nearly
// every relaxation targets another partition. With one query per warp, each
// such relaxation reads one 4-byte value from a random place in HBM, and the
// memory system moves a whole 32- to 64-byte granule for it. Here the state of
// a group is vertex-major, D[group][v][0..G), so the G values of one vertex
// share one line: a relaxation of arc (v, u) is done for every query of the
// group at once, and one line transfer serves G lanes. The partition's CSR
// (row offsets, targets, weights) is likewise read once per (partition, group)
// visit for all G queries (the sharing of Sec. 3.2 and App. B.1, with the
// buckets keyed by (partition, group): K = |Q| / G).
//
// Rounds (one persistent cooperative launch, two device-wide barriers each):
//   SCAN     collect work items: every (partition, group) whose dirty flag was
//            set in the previous round, and every pending hub vertex (more than
//            hub_min arcs) cut into chunks of at most hub_chunk arcs
//   PROCESS  each block claims items. A partition item stages the partition's
//            row offsets and its pending masks into shared memory with one 1-D
//            TMA bulk phase, lists the pending vertices and relaxes their arcs
//            for the lanes marked pending; a hub chunk relaxes one range of a
//            hub's arcs.
// Arcs are relaxed 32 at a time per warp, one arc per lane: the lane copies
// its arc's target line (the G current values) into the warp's shared memory
// with 16-byte cp.async copies, two such steps in flight, while the lanes of
// each query compare the previous step's values with their new ones.
//
// Operations for other partitions are consolidated where they land (Sec. 4.2
// with one slot per (query, vertex)): a relaxation that lowers the target's
// value writes it with atomicMin and marks the target in the next round's
// pending mask of its (partition, group), together with the dirty flag that
// schedules it. Values only decrease and every decrease schedules a later
// expansion, so the distances reached are exact whatever the order.
//
// Round r reads pend[r & 1] and dirty[r & 1] and writes pend[(r + 1) & 1] and
// dirty[(r + 1) & 1]; a (partition, group)'s masks of round r are cleared by
// its visit, a hub's by the scan, so both halves are zero again when reused.
#include <cstdio>

#include "fg_device.cuh"

namespace fg {

constexpr int kGThreads = 256;
constexpr int kGWarps = kGThreads / 32;
constexpr int kGUnroll = 8;  // arc slots per lane group compared per inner step

// Shared memory of one block: the item buffers, then per warp two [32][G]
// step buffers of target lines and one [32][G] table of source values.
__host__ __device__ inline size_t group_item_words(int S) { return (size_t)(S + 4) * 2 + (size_t)S * 2; }
__host__ __device__ inline size_t group_warp_words(int G) { return (size_t)3 * 32u * (size_t)G; }
__host__ __device__ inline size_t group_smem_bytes(int S, int G) {
  return (group_item_words(S) + (size_t)kGWarps * group_warp_words(G)) * sizeof(uint32_t);
}

__device__ __forceinline__ uint32_t g_relax(Ctrl *c, uint32_t d, uint32_t w) {
  const uint64_t s = (uint64_t)d + (uint64_t)w;
  if (s >= (uint64_t)kInf) {
    atomicCAS(&c->status, 0, (int)FG_ERR_OVERFLOW);
    return kInf - 1u;
  }
  return (uint32_t)s;
}

// Block-wide exclusive scan of one u64 per thread (kGThreads threads).
__device__ __forceinline__ unsigned long long g_block_scan(unsigned long long x, unsigned long long *s_warp,
                                                           unsigned long long &total) {
  const int lane = lane_id(), wid = threadIdx.x >> 5;
  const unsigned long long incl = warp_incl_scan(x);
  if (lane == 31) s_warp[wid] = incl;
  block_sync();
  if (wid == 0) {
    const unsigned long long v = lane < kGWarps ? s_warp[lane] : 0ull;
    const unsigned long long vi = warp_incl_scan(v);
    if (lane < kGWarps) s_warp[lane] = vi - v;
    if (lane == kGWarps - 1) s_warp[kGWarps] = vi;
  }
  block_sync();
  const unsigned long long ex = s_warp[wid] + incl - x;
  total = s_warp[kGWarps];
  block_sync();
  return ex;
}

// One step's arcs: lane l holds arc l (target u, weight w, owner o = row of the
// warp's source-value table, has = the arc exists).
struct ArcStep {
  uint32_t u, w, o;
  bool has;
};

// The lane copies its arc's target line (G values, G / 4 copies of 16 bytes)
// into row `lane` of the step buffer, and closes the step's copy group.
__device__ __forceinline__ void g_issue(const ArcStep &s, uint32_t *buf, const uint32_t *Dg, int G, int glog2,
                                        int lane) {
  if (s.has) {
    const uint32_t *src = Dg + ((size_t)s.u << glog2);
    uint32_t *dst = buf + ((uint32_t)lane << glog2);
    for (int k = 0; k < G; k += 4) cp_async16_cg(dst + k, src + k);
  }
  cp_async_commit();
}

// Compare and lower. Lane (h, g) takes arc slot sl = j * SL + h and query g:
// its source value (from sdv[owner][g], or dv_own for a hub chunk), the new
// value through the arc, and the target's value copied into buf[sl][g] (a
// snapshot: values only decrease, so an older value is an upper bound and can
// only let a useless write through). Lanes whose new value is smaller write it
// with atomicMin and mark the target pending for the next round.
template <int QT>
__device__ __forceinline__ void g_process(const GroupArgs &a, const ArcStep &s, const uint32_t *buf,
                                          const uint32_t *sdv, uint32_t dv_own, uint32_t *Dg, uint32_t *pend_g,
                                          uint32_t *dirty_g, uint32_t *gbest_n, int g, int h, int SL,
                                          unsigned long long &relaxed, unsigned long long &improved) {
  const int G_ = a.G;
  const unsigned gmask = G_ == 32 ? 0xFFFFFFFFu : ((1u << G_) - 1u);
  const int slog2 = a.g.slog2;
  for (int j0 = 0; j0 < 32; j0 += SL * kGUnroll) {
#pragma unroll
    for (int q = 0; q < kGUnroll; ++q) {
      const int sl = j0 + q * SL + h;  // < 32: 32 is a multiple of SL * kGUnroll
      const uint32_t uu = __shfl_sync(kFull, s.u, sl);
      const uint32_t ww = __shfl_sync(kFull, s.w, sl);
      const uint32_t oo = __shfl_sync(kFull, s.o, sl);
      const bool hh = __shfl_sync(kFull, s.has ? 1u : 0u, sl) != 0u;
      uint32_t dv = kInf;
      if (hh) dv = sdv != nullptr ? sdv[(oo << a.glog2) + (uint32_t)g] : dv_own;
      const bool act = hh && dv != kInf;
      const uint32_t nd = act ? g_relax(a.ctrl, dv, QT == Q_BFS ? 1u : ww) : kInf;
      const uint32_t cur = act ? buf[((uint32_t)sl << a.glog2) + (uint32_t)g] : 0u;
      const bool imp = act && nd < cur;
      relaxed += act ? 1ull : 0ull;
      if (imp) atomicMin(Dg + ((size_t)uu << a.glog2) + (size_t)g, nd);
      const unsigned im = __ballot_sync(kFull, imp);
      const unsigned mine = (im >> (h * G_)) & gmask;
      if (mine != 0u && g == 0) {
        atomicOr(pend_g + uu, mine);
        dirty_g[uu >> slog2] = 1u;
        improved += (unsigned long long)__popc(mine);
      }
      if (gbest_n != nullptr) {
        // smallest new value of the group, for the next round's window
        const uint32_t mn = __reduce_min_sync(kFull, imp ? nd : kInf);
        if (mn != kInf && (threadIdx.x & 31) == 0) atomicMin(gbest_n, mn);
      }
    }
  }
}

// Relax a sequence of nsteps steps of 32 arcs, the copies of step i + 1 in
// flight while step i is compared. make(i) fills a step (warp-collective).
template <int QT, typename Make>
__device__ __forceinline__ void g_run_steps(const GroupArgs &a, uint32_t nsteps, Make make, uint32_t *wbuf,
                                            const uint32_t *sdv, uint32_t dv_own, uint32_t *Dg, uint32_t *pend_g,
                                            uint32_t *dirty_g, uint32_t *gbest_n, int g, int h, int SL, int lane,
                                            unsigned long long &relaxed, unsigned long long &improved,
                                            unsigned long long &arcs) {
  if (nsteps == 0u) return;
  const int G_ = a.G;
  uint32_t *buf[2] = {wbuf, wbuf + 32 * G_};
  ArcStep cur = make(0u);
  g_issue(cur, buf[0], Dg, G_, a.glog2, lane);
  for (uint32_t i = 0; i < nsteps; ++i) {
    ArcStep nxt{0u, 0u, 0u, false};
    if (i + 1u < nsteps) {
      nxt = make(i + 1u);
      g_issue(nxt, buf[(i + 1u) & 1u], Dg, G_, a.glog2, lane);
    } else {
      cp_async_commit();  // an empty group keeps "all but the newest group" meaning step i
    }
    cp_async_wait<1>();
    __syncwarp();
    arcs += cur.has ? 1ull : 0ull;
    g_process<QT>(a, cur, buf[i & 1u], sdv, dv_own, Dg, pend_g, dirty_g, gbest_n, g, h, SL, relaxed, improved);
    __syncwarp();  // buf[i & 1] is refilled by step i + 2
    cur = nxt;
  }
  cp_async_wait<0>();
}

template <int QT>
__global__ void __launch_bounds__(kGThreads, 2) group_kernel(GroupArgs a) {
  extern __shared__ __align__(16) uint32_t g_smem[];
  __shared__ __align__(8) uint64_t s_bar;
  __shared__ unsigned long long s_scan[kGWarps + 1];
  __shared__ uint32_t s_item, s_batch, s_cnt;
  const int lane = lane_id(), wid = threadIdx.x >> 5;
  const DevGraph &G = a.g;
  const int S = G.S;
  const int Gq = a.G;
  const int g = lane & (Gq - 1);     // query of the group held by this lane
  const int h = lane >> a.glog2;     // arc slot of this lane
  const int SL = 32 >> a.glog2;      // arc slots per warp
  uint32_t *s_rp = g_smem;           // [S + 4] row offsets of the item's partition
  uint32_t *s_pm = s_rp + (S + 4);   // [S]     pending masks of the item's group
  uint32_t *s_vid = s_pm + S;        // [S]     pending vertices (partition-local), listed
  uint32_t *s_pre = s_vid + S;       // [S + 4] exclusive prefix of their arc counts
  uint32_t *wbuf = s_pre + (S + 4) + (size_t)wid * group_warp_words(Gq);  // 2 x [32][G] step buffers
  uint32_t *sdv = wbuf + 64 * Gq;                                          // [32][G] source values
  Ctrl *c = a.ctrl;
  unsigned gen = *reinterpret_cast<volatile unsigned *>(&c->bar_gen);
  uint32_t phase = 0;
  unsigned long long n_relaxed = 0, n_improved = 0, n_visits = 0, n_arcs = 0;
  uint64_t t_prev = (blockIdx.x == 0 && threadIdx.x == 0) ? global_ns() : 0ull;
  unsigned long long ph[6] = {0ull, 0ull, 0ull, 0ull, 0ull, 0ull};
#define FG_GPHASE(k)                                            \
  do {                                                          \
    if (blockIdx.x == 0 && threadIdx.x == 0) {                  \
      const uint64_t t_now = global_ns();                       \
      ph[k] += t_now - t_prev;                                  \
      t_prev = t_now;                                           \
    }                                                           \
  } while (0)

  if (threadIdx.x == 0) {
    mbar_init(&s_bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    fence_proxy_async_smem();
  }
  block_sync();

  const uint64_t K = (uint64_t)a.ngroups * (uint64_t)G.nparts;
  const uint64_t tid = (uint64_t)blockIdx.x * kGThreads + threadIdx.x, nthr = (uint64_t)gridDim.x * kGThreads;
  const size_t row = (size_t)a.npad;  // vertices per group row

  // ---- K0: state and masks (InitBuffers, first half) ----
  {
    const uint64_t dwords = (uint64_t)a.ngroups * (uint64_t)a.npad * (uint64_t)Gq;
    for (uint64_t i = tid; i < dwords / 4u; i += nthr)
      reinterpret_cast<uint4 *>(a.D)[i] = make_uint4(kInf, kInf, kInf, kInf);
    const uint64_t pwords = 2ull * (uint64_t)a.ngroups * (uint64_t)a.npad;
    for (uint64_t i = tid; i < pwords / 4u; i += nthr) reinterpret_cast<uint4 *>(a.pend)[i] = make_uint4(0u, 0u, 0u, 0u);
    for (uint64_t i = tid; i < 2ull * K; i += nthr) a.dirty[i] = 0u;
    if (a.gbest)
      for (uint64_t i = tid; i < 2ull * (uint64_t)a.ngroups; i += nthr) a.gbest[i] = kInf;
  }
  if (!grid_barrier(c, gen, a.watchdog_ns)) goto done;
  FG_GPHASE(0);

  // ---- INIT: each query's source gets value 0 and is pending in round 0 ----
  for (uint64_t q = tid; q < (uint64_t)a.nq; q += nthr) {
    const int32_t s = a.src[q];
    if (s < 0 || s >= G.n) {
      raise_status(c, FG_ERR_INVALID_ARG, kSiteSource);
      continue;
    }
    const uint32_t v = G.intl ? (uint32_t)G.intl[s] : (uint32_t)s;
    const uint32_t grp = (uint32_t)(q >> a.glog2), gq = (uint32_t)(q & (uint64_t)(Gq - 1));
    a.D[((size_t)grp * row + v) * (size_t)Gq + gq] = 0u;
    atomicOr(a.pend + (size_t)grp * row + v, 1u << gq);
    a.dirty[(size_t)grp * G.nparts + (v >> G.slog2)] = 1u;
    if (a.gbest) atomicMin(a.gbest + grp, 0u);
  }
  if (!grid_barrier(c, gen, a.watchdog_ns)) goto done;
  FG_GPHASE(1);

  for (uint32_t round = 0;; ++round) {
    const uint32_t cur = round & 1u, nxt = cur ^ 1u;
    uint32_t *pend_c = a.pend + (size_t)cur * (size_t)a.ngroups * row;
    uint32_t *pend_n = a.pend + (size_t)nxt * (size_t)a.ngroups * row;
    uint32_t *dirty_c = a.dirty + (size_t)cur * K;
    uint32_t *dirty_n = a.dirty + (size_t)nxt * K;
    // ---- SCAN: hub chunks, then dirty (partition, group) items ----
    {
      if (blockIdx.x == 0 && threadIdx.x == 0) {
        c->g_hub_items[nxt] = 0u;
        c->g_items[nxt] = 0u;
        c->g_next[nxt] = 0u;
      }
      if (a.gbest)
        for (uint64_t i = tid; i < (uint64_t)a.ngroups; i += nthr) a.gbest[(size_t)nxt * a.ngroups + i] = kInf;
      const uint64_t HK = (uint64_t)a.nhubs * (uint64_t)a.ngroups;
      for (uint64_t k = tid; k < HK; k += nthr) {
        const uint32_t grp = (uint32_t)(k / (uint64_t)a.nhubs), hi = (uint32_t)(k % (uint64_t)a.nhubs);
        const uint32_t v = a.hubs[hi];
        uint32_t *pw = pend_c + (size_t)grp * row + v;
        const uint32_t m = __ldcg(pw);
        if (m == 0u) continue;
        *pw = 0u;
        const uint32_t e0 = G.rp[v], e1 = G.rp[v + 1];
        const uint32_t nch = (e1 - e0 + a.hub_chunk - 1u) / a.hub_chunk;
        const uint32_t b = atomicAdd(&c->g_hub_items[cur], nch);
        for (uint32_t ch = 0; ch < nch && b + ch < a.hub_cap; ++ch)
          a.items[b + ch] = make_uint4(grp, v, e0 + ch * a.hub_chunk, m);
        if (b + nch > a.hub_cap) raise_status(c, FG_ERR_BIN_OVERFLOW, kSiteArena);
      }
      const uint64_t gw = tid >> 5, nw = nthr >> 5;
      for (uint64_t k0 = gw * 32ull; k0 < K; k0 += nw * 32ull) {
        const uint64_t k = k0 + (uint64_t)lane;
        bool act = false;
        if (k < K) {
          act = __ldcg(dirty_c + k) != 0u;
          if (act) dirty_c[k] = 0u;
        }
        const unsigned m = __ballot_sync(kFull, act);
        if (m == 0u) continue;
        uint32_t b = 0;
        if (lane == 0) b = atomicAdd(&c->g_items[cur], (unsigned)__popc(m));
        b = __shfl_sync(kFull, b, 0);
        if (act) a.items[a.hub_cap + b + __popc(m & ((1u << lane) - 1u))] = make_uint4((uint32_t)k, 0u, 0u, 0u);
      }
    }
    if (!grid_barrier(c, gen, a.watchdog_ns)) goto done;
    FG_GPHASE(2);
    const uint32_t n_hub = umin64(*reinterpret_cast<volatile unsigned *>(&c->g_hub_items[cur]), a.hub_cap);
    const uint32_t n_reg = *reinterpret_cast<volatile unsigned *>(&c->g_items[cur]);
    if (n_hub + n_reg == 0u) break;
    if (round >= a.max_rounds) {
      if (threadIdx.x == 0) raise_status(c, FG_ERR_TIMEOUT, kSiteRounds);
      break;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      c->rounds += 1ull;
      if ((unsigned long long)n_hub + n_reg > c->max_round_ops) c->max_round_ops = (unsigned long long)n_hub + n_reg;
    }
    const uint32_t bound_w = a.window;
    // ---- PROCESS ----
    for (;;) {
      if (threadIdx.x == 0) {
        uint32_t idx = atomicAdd(&c->g_next[cur], 1u);
        if (ld_volatile_i32(&c->abort)) idx = n_hub + n_reg;
        s_item = idx;
        s_batch = 0u;
      }
      block_sync();
      const uint32_t idx = s_item;
      if (idx >= n_hub + n_reg) break;
      if (idx < n_hub) {
        // -- one chunk of a hub's arcs, for the lanes pending on it --
        const uint4 it = __ldcg(a.items + idx);
        const uint32_t grp = it.x, v = it.y, eb = it.z, m = it.w;
        const uint32_t e1 = G.rp[v + 1];
        const uint32_t ee = eb + a.hub_chunk < e1 ? eb + a.hub_chunk : e1;
        uint32_t *Dg = a.D + (size_t)grp * row * (size_t)Gq;
        uint32_t dv = kInf;
        if (((m >> g) & 1u) != 0u) dv = __ldcg(Dg + ((size_t)v << a.glog2) + (size_t)g);
        uint32_t *gb_n = a.gbest ? a.gbest + (size_t)nxt * a.ngroups + grp : nullptr;
        // the warp takes steps wid, wid + 8, ... of 32 consecutive arcs
        const uint32_t total = ee - eb;
        const uint32_t all_steps = (total + 31u) / 32u;
        const uint32_t my_steps = all_steps > (uint32_t)wid ? (all_steps - 1u - (uint32_t)wid) / kGWarps + 1u : 0u;
        auto make = [&](uint32_t i) {
          ArcStep st;
          const uint32_t e = eb + ((uint32_t)wid + i * kGWarps) * 32u + (uint32_t)lane;
          st.has = e < ee;
          st.u = st.has ? __ldg(G.adj + e) : 0u;
          st.w = (st.has && QT != Q_BFS && G.wt != nullptr) ? __ldg(G.wt + e) : 1u;
          st.o = 0u;
          return st;
        };
        g_run_steps<QT>(a, my_steps, make, wbuf, nullptr, dv, Dg, pend_n + (size_t)grp * row,
                        dirty_n + (size_t)grp * G.nparts, gb_n, g, h, SL, lane, n_relaxed, n_improved, n_arcs);
        if (threadIdx.x == 0) ++n_visits;
        block_sync();
        continue;
      }
      // -- a (partition, group) item --
      const uint4 it = __ldcg(a.items + a.hub_cap + (idx - n_hub));
      const uint32_t key = it.x;
      const uint32_t grp = key / (uint32_t)G.nparts, p = key - grp * (uint32_t)G.nparts;
      const uint32_t base = p << G.slog2;
      uint32_t *pm_g = pend_c + (size_t)grp * row + base;
      // 1. stage the partition's row offsets and the group's pending masks
      //    (one bulk phase; the expected bytes are announced before the copies)
      if (threadIdx.x == 0) {
        const uint32_t b_rp = (uint32_t)(S + 4) * 4u, b_pm = (uint32_t)S * 4u;
        fence_proxy_async_smem();
        mbar_arrive_expect_tx(&s_bar, b_rp + b_pm);
        bulk_g2s(s_rp, G.rp + base, b_rp, &s_bar);
        bulk_g2s(s_pm, pm_g, b_pm, &s_bar);
      }
      {
        // the outcome is made block-uniform, so no thread leaves the item alone
        const int ok = __syncthreads_and(mbar_wait(&s_bar, phase, a.watchdog_ns) ? 1 : 0);
        if (!ok) {
          if (threadIdx.x == 0) {
            raise_status(c, FG_ERR_TIMEOUT, kSiteStage);
            (void)mbar_wait(&s_bar, phase, 1000000ull);  // the copies in flight, once more, bounded
          }
          block_sync();
          break;
        }
      }
      phase ^= 1u;
      // 2. this round's masks of the item are taken: clear them for reuse
      for (int i = threadIdx.x; i < (S >> 2); i += kGThreads)
        reinterpret_cast<uint4 *>(pm_g)[i] = make_uint4(0u, 0u, 0u, 0u);
      uint32_t *Dg = a.D + (size_t)grp * row * (size_t)Gq;
      uint32_t *gb_n = a.gbest ? a.gbest + (size_t)nxt * a.ngroups + grp : nullptr;
      // 3. window (Delta-stepping across rounds): lanes whose value is at or
      //    beyond the group's bound stay pending for a later round
      if (bound_w != 0u && a.gbest != nullptr) {
        const uint32_t bound = sat_add_u32(__ldcg(a.gbest + (size_t)cur * a.ngroups + grp), bound_w);
        for (int i0 = wid * SL; i0 < S; i0 += kGWarps * SL) {
          const int i = i0 + h;
          const uint32_t m = s_pm[i];
          bool def = false;
          uint32_t dv = kInf;
          if (((m >> g) & 1u) != 0u) {
            dv = __ldcg(Dg + ((size_t)(base + (uint32_t)i) << a.glog2) + (size_t)g);
            def = dv >= bound;
          }
          const unsigned dm = __ballot_sync(kFull, def);
          const unsigned gmask = Gq == 32 ? 0xFFFFFFFFu : ((1u << Gq) - 1u);
          const unsigned mine = (dm >> (h * Gq)) & gmask;
          const uint32_t mn = __reduce_min_sync(kFull, def ? dv : kInf);
          if (mine != 0u && g == 0) {
            atomicOr(pend_n + (size_t)grp * row + base + (uint32_t)i, mine);
            dirty_n[(size_t)grp * G.nparts + p] = 1u;
            s_pm[i] = m & ~mine;
          }
          if (mn != kInf && lane == 0) atomicMin(gb_n, mn);
        }
        block_sync();
      }
      // 4. list the pending vertices and the exclusive prefix of their arcs
      {
        const int per = (S + kGThreads - 1) / kGThreads;
        unsigned long long x = 0;
        for (int j = 0; j < per; ++j) {
          const int i = threadIdx.x * per + j;
          if (i < S && s_pm[i] != 0u) {
            const uint32_t deg = s_rp[i + 1] - s_rp[i];
            if (deg > 0u) x += (1ull << 32) | (unsigned long long)deg;
          }
        }
        unsigned long long tot;
        unsigned long long ex = g_block_scan(x, s_scan, tot);
        for (int j = 0; j < per; ++j) {
          const int i = threadIdx.x * per + j;
          if (i < S && s_pm[i] != 0u) {
            const uint32_t deg = s_rp[i + 1] - s_rp[i];
            if (deg > 0u) {
              const uint32_t pos = (uint32_t)(ex >> 32);
              s_vid[pos] = (uint32_t)i;
              s_pre[pos] = (uint32_t)ex;
              ex += (1ull << 32) | (unsigned long long)deg;
            }
          }
        }
        if (threadIdx.x == 0) {
          s_cnt = (uint32_t)(tot >> 32);
          s_pre[tot >> 32] = (uint32_t)tot;
        }
        block_sync();
      }
      const uint32_t nv = s_cnt;
      // 5. relax: warps take batches of up to 32 listed vertices; the batch's
      //    arcs are cut into steps of 32 (merge path over the batch's lanes)
      for (;;) {
        uint32_t b0 = 0;
        if (lane == 0) b0 = atomicAdd(&s_batch, 32u);
        b0 = __shfl_sync(kFull, b0, 0);
        if (b0 >= nv) break;
        const uint32_t j = b0 + (uint32_t)lane;
        const bool valid = j < nv;
        const uint32_t li = valid ? s_vid[j] : 0u;
        const uint32_t m = valid ? s_pm[li] : 0u;
        const uint32_t a0 = valid ? s_rp[li] : 0u;
        const uint32_t deg = valid ? s_rp[li + 1] - a0 : 0u;
        const uint32_t incl = warp_incl_scan(deg);
        const uint32_t exd = incl - deg;
        const uint32_t tot = __shfl_sync(kFull, incl, 31);
        // the batch's source values, fresh from L2 (the pending bit was set
        // because the value fell; an older copy could miss that fall): row L
        // of sdv holds vertex L's values of the group, kInf where not pending
        for (int L0 = 0; L0 < 32; L0 += SL) {
          const int L = L0 + h;
          const uint32_t vL = __shfl_sync(kFull, li, L);
          const uint32_t mL = __shfl_sync(kFull, m, L);
          uint32_t d = kInf;
          if (((mL >> g) & 1u) != 0u) d = __ldcg(Dg + ((size_t)(base + vL) << a.glog2) + (size_t)g);
          sdv[(L << a.glog2) + g] = d;
        }
        __syncwarp();
        auto make = [&](uint32_t i) {
          ArcStep st;
          const uint32_t t = i * 32u + (uint32_t)lane;
          st.has = t < tot;
          const int L = owner_lane(exd, st.has ? t : 0u);
          const uint32_t eL = __shfl_sync(kFull, a0, L) + (t - __shfl_sync(kFull, exd, L));
          st.u = st.has ? __ldg(G.adj + eL) : 0u;
          st.w = (st.has && QT != Q_BFS && G.wt != nullptr) ? __ldg(G.wt + eL) : 1u;
          st.o = (uint32_t)L;
          return st;
        };
        g_run_steps<QT>(a, (tot + 31u) / 32u, make, wbuf, sdv, kInf, Dg, pend_n + (size_t)grp * row,
                        dirty_n + (size_t)grp * G.nparts, gb_n, g, h, SL, lane, n_relaxed, n_improved, n_arcs);
        __syncwarp();  // sdv is rewritten by the next batch
      }
      if (threadIdx.x == 0) ++n_visits;
      block_sync();  // shared buffers and s_item are reused by the next item
    }
    if (!grid_barrier(c, gen, a.watchdog_ns)) goto done;
    FG_GPHASE(5);
  }
done:
#undef FG_GPHASE
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    ph[2] += global_ns() - t_prev;
    for (int k = 0; k < 6; ++k) atomicAdd(&c->phase_ns[k], ph[k]);
  }
  {
    const unsigned long long r = warp_sum(n_relaxed), im = warp_sum(n_improved), ar = warp_sum(n_arcs);
    if (lane == 0) {
      atomicAdd(&c->edges, r);
      atomicAdd(&c->ops, im);
      atomicAdd(&c->arcs_read, ar);
    }
    if (threadIdx.x == 0) atomicAdd(&c->visits, n_visits);
  }
}

// D[group][v][g] (internal order) -> out[group * G + g][orig(v)] for v < n.
// A block moves 32 vertices of one group: 32 * G words read as whole lines,
// transposed in shared memory, written as G runs of 32 values.
__global__ void __launch_bounds__(256) group_out_kernel(const uint32_t *D, uint32_t *out, const int32_t *orig,
                                                        int64_t n, int64_t npad, int32_t G, int32_t glog2,
                                                        int32_t nq, int64_t tiles_per_group) {
  __shared__ uint32_t t[32][33];
  const int64_t grp = blockIdx.x / tiles_per_group;
  const int64_t v0 = (blockIdx.x % tiles_per_group) * 32;
  const uint32_t *src = D + ((size_t)grp * (size_t)npad + (size_t)v0) * (size_t)G;
  for (int i = threadIdx.x; i < 32 * G; i += blockDim.x) {
    const int vl = i >> glog2, gq = i & (G - 1);
    t[gq][vl] = (v0 + vl < n) ? src[i] : kInf;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 32 * G; i += blockDim.x) {
    const int gq = i >> 5, vl = i & 31;
    const int64_t q = grp * G + gq, v = v0 + vl;
    if (q < nq && v < n) {
      const int64_t o = orig ? (int64_t)orig[v] : v;
      out[q * n + o] = t[gq][vl];
    }
  }
}

static const void *group_fn(int qtype) {
  return qtype == Q_BFS ? (const void *)group_kernel<Q_BFS> : (const void *)group_kernel<Q_SSSP>;
}

cudaError_t group_grid_size(int S, int G, int *blocks, int *threads, size_t *smem) {
  *threads = kGThreads;
  *smem = group_smem_bytes(S, G);
  int best = 1 << 30, dev = 0, sms = 0;
  cudaError_t e;
  for (int qt = 0; qt < 2; ++qt) {
    const void *fn = group_fn(qt);
    if ((e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)*smem)) != cudaSuccess)
      return e;
    int per_sm = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kGThreads, *smem)) != cudaSuccess)
      return e;
    best = per_sm < best ? per_sm : best;
  }
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  if (best < 1) return cudaErrorInvalidConfiguration;
  *blocks = best * sms;
  return cudaSuccess;
}

cudaError_t launch_group(const GroupArgs &a, int blocks, int threads, size_t smem, cudaStream_t s) {
  GroupArgs copy = a;
  void *args[] = {(void *)&copy};
  return cudaLaunchCooperativeKernel(group_fn(a.qtype), dim3(blocks), dim3(threads), args, smem, s);
}

cudaError_t launch_group_out(const GroupArgs &a, uint32_t *out, cudaStream_t s) {
  const int64_t n = a.g.n;
  const int64_t tiles = (n + 31) / 32;
  const int64_t grid = tiles * (int64_t)a.ngroups;
  if (grid <= 0) return cudaSuccess;
  group_out_kernel<<<(unsigned)grid, 256, 0, s>>>(a.D, out, a.g.orig, n, a.npad, a.G, a.glog2, a.nq, tiles);
  return cudaGetLastError();
}

}  // namespace fg
