// Group engine: the buffered loop of Alg. 2 for SSSP and BFS with queries
// processed in groups of G (8, 16, 32 or 64; one query per lane, two for 64).
//
// Why groups. On graphs whose partitions are cut by almost every arc (power-law
// graphs with the paper's random equal-vertex partitions, Sec. 6.1), nearly
// every relaxation targets another partition. With one query per warp, each
// such relaxation reads one 4-byte value from a random place in HBM, and the
// memory system moves a whole 32- to 64-byte granule for it. Here the state of
// a group is vertex-major, D[group][v][0..G), so the G values of one vertex
// share one line: a relaxation of arc (v, u) is done for every query of the
// group at once, and one line access serves G lanes. The partition's CSR (row
// offsets, targets, weights) is likewise read once per (partition, group)
// visit for all G queries (the sharing of Sec. 3.2 and App. B.1, with the
// buckets keyed by (partition, group): K = |Q| / G).
//
// Rounds (one persistent cooperative launch, two device-wide barriers each):
//   SCAN     collect work items: every (partition, group) whose dirty flag was
//            set in the previous round, and every pending hub vertex (more than
//            kHubMin arcs) cut into chunks of at most hub_chunk arcs
//   PROCESS  in each block, one producer warp claims items, stages a partition
//            item's row offsets and pending masks into one of two shared-memory
//            buffers with a 1-D TMA bulk phase, lists the pending vertices and
//            publishes the item; eight consumer warps take batches of the
//            published item (32 listed vertices, or 32 arcs of a hub chunk)
//            and move on to the other buffer's item when it runs out, so no
//            warp waits for the others between items. Each buffer has a "full"
//            barrier (the producer's arrival) and an "empty" barrier (one
//            arrival per consumer warp) that gate its reuse.
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
//
// Three relaxation forms share this loop. Dense (SSSP): the warp reads a
// target's line for each arc and every pending lane compares its value.
// Sparse (SSSP, a vertex with at most kSparseT pending lanes): each lane
// takes one (arc, query) pair and reads that single value. Bitwise (BFS):
// rounds are levels, so a lane takes one arc and sets the source's frontier
// lanes in the target's reach mask; the lanes that were new get their level.
// The host orders a batch's queries before it cuts them into groups, by
// two-hop reach, or by source position on road-like graphs, so that the
// queries of a group advance alike.
#include <cstdio>
#include <type_traits>

#include "fg_device.cuh"

namespace fg {

constexpr int kGCons = 8;                    // consumer warps per block
constexpr int kGThreads = (kGCons + 1) * 32;  // and one producer warp
constexpr int kGUnroll = 8;                  // arc slots per lane group with loads in flight at once
constexpr int kGUnroll64 = 8;                // the same for groups of 64 (two values per lane)

enum : uint32_t { kItemPart = 0, kItemHub = 1, kItemEnd = 2 };

// A published item (one per buffer).
struct ItemDesc {
  uint32_t kind;  // kItemPart, kItemHub or kItemEnd (no more items this round)
  uint32_t grp;   // group
  uint32_t pv;    // partition (kItemPart) or hub vertex (kItemHub)
  uint32_t n;     // listed vertices (kItemPart) or steps of 32 arcs (kItemHub)
  uint32_t eb, ee;  // hub chunk: arc range
  uint32_t next;  // claim counter of the consumers (vertices or steps)
  uint32_t ns;    // kItemPart: listed sparse vertices (few pending lanes)
  uint32_t next_s;  // claim counter of the sparse vertices
  uint32_t pad;
  unsigned long long m;  // hub chunk: the lanes pending on the hub
};

// A listed vertex with at most kSparseT pending lanes is relaxed pair by pair:
// a lane takes one (arc, pending query) pair and reads that query's 4-byte
// value of the target, instead of the warp reading the target's whole line
// for every arc. Lanes map to kSparseT slots per arc (32 / kSparseT arcs per
// warp step).
constexpr int kSparseT = 4;

// Lane layout by group size. G <= 32: lane (h, g) holds query g of the group
// for arc slot h (SL = 32 / G arcs per warp step), and a vertex's pending
// lanes are a 32-bit mask. G = 64: lane l holds queries 2l and 2l + 1 (one
// 8-byte pair of the vertex's line), one arc per warp step, and the mask is 64
// bits with query 2l + j at bit 32j + l, so that a warp ballot per half is a
// mask word.
template <int GQ>
struct GroupLanes {
  using M = uint32_t;
  static constexpr int SL = 32 / GQ;
};
template <>
struct GroupLanes<64> {
  using M = unsigned long long;
  static constexpr int SL = 1;
};
template <int GQ>
__host__ __device__ __forceinline__ typename GroupLanes<GQ>::M group_bit(uint32_t gq) {
  if constexpr (GQ == 64) return 1ull << (((gq & 1u) << 5) | (gq >> 1));
  else return 1u << gq;
}

// Shared memory: two item buffers (row offsets, pending masks of one or two
// words, listed vertices), then per consumer warp the current step's 32 arcs
// (uint4 each) and one [B][G] table of source values, B = the listed
// vertices a warp takes at a time (32; 16 for G = 64, so that three blocks
// fit an SM).
__host__ __device__ constexpr int group_batch(int G) { return G == 64 ? 16 : 32; }
__host__ __device__ inline size_t group_mask_words(int G) { return G == 64 ? 2u : 1u; }
__host__ __device__ inline size_t group_item_words(int S, int G) {
  return (size_t)(S + 4) + (size_t)S * (1u + group_mask_words(G));
}
__host__ __device__ inline size_t group_smem_bytes(int S, int G) {
  return (2 * group_item_words(S, G) + (size_t)kGCons * (128u + (size_t)group_batch(G) * (size_t)G)) *
         sizeof(uint32_t);
}

__device__ __forceinline__ uint32_t g_relax(Ctrl *c, uint32_t d, uint32_t w) {
  const uint64_t s = (uint64_t)d + (uint64_t)w;
  if (s >= (uint64_t)kInf) {
    atomicCAS(&c->status, 0, (int)FG_ERR_OVERFLOW);
    return kInf - 1u;
  }
  return (uint32_t)s;
}

__host__ __device__ constexpr int ilog2c(int x) { return x <= 1 ? 0 : 1 + ilog2c(x / 2); }

// One step of up to 32 arcs, staged by the warp in sarc[0..32): target, weight,
// owner row (kNoArc: no arc in this slot). The arcs are relaxed SL = 32 / GQ at
// a time, one per lane group, kGUnroll groups in flight: each lane reads its
// query's current value of the target (a plain load: values only decrease, so
// a stale copy is an upper bound and can only let a useless write through),
// and only lanes whose new value is smaller lower it with a fire-and-forget
// atomicMin; one lane per lane group then marks the target pending for the
// next round. The source value of lane g is sdv_g[owner * GQ] (sdv_g = the
// warp's [32][GQ] table + g; kInf: lane not pending), or dv_own when sdv_g is
// null (a hub chunk: one source vertex). Dg_g = the group's state + g.
constexpr uint32_t kNoArc = 0xFFFFFFFFu;

template <int QT, int GQ>
__device__ __forceinline__ void g_step(const GroupArgs &a, const uint4 *sarc, const uint32_t *sdv_g,
                                       uint32_t dv_own, uint32_t *Dg_g, uint32_t *pend_g, uint32_t *dirty_g,
                                       uint32_t *gbest_n, int g, int h, uint32_t &improved,
                                       uint32_t &lanes_marked, bool chk) {
  constexpr int LG = ilog2c(GQ), SL = 32 / GQ;
  constexpr unsigned GM = GQ == 32 ? 0xFFFFFFFFu : ((1u << GQ) - 1u);
  const int slog2 = a.g.slog2;
#pragma unroll 1
  for (int j0 = 0; j0 < 32; j0 += SL * kGUnroll) {
    uint32_t nd[kGUnroll], cur[kGUnroll];
    bool act[kGUnroll];
#pragma unroll
    for (int q = 0; q < kGUnroll; ++q) {
      const uint4 e = sarc[j0 + q * SL + h];  // one broadcast read per lane group
      uint32_t dv = kInf;
      if (e.z != kNoArc) dv = sdv_g != nullptr ? sdv_g[e.z << LG] : dv_own;
      act[q] = dv != kInf;
      uint32_t sum = dv + (QT == Q_BFS ? 1u : e.y);
      if (QT != Q_BFS && chk && act[q] && (sum < dv || sum == kInf)) {  // 2^32 - 1 reached: saturate and report
        atomicCAS(&a.ctrl->status, 0, (int)FG_ERR_OVERFLOW);
        sum = kInf - 1u;
      }
      nd[q] = sum;
      cur[q] = act[q] ? Dg_g[(size_t)e.x << LG] : 0u;
    }
#pragma unroll
    for (int q = 0; q < kGUnroll; ++q) {
      const bool imp = act[q] && nd[q] < cur[q];
      const uint32_t uq = sarc[j0 + q * SL + h].x;  // read again rather than held in a register
      if (imp) atomicMin(Dg_g + ((size_t)uq << LG), nd[q]);
      const unsigned im = __ballot_sync(kFull, imp);
      if (im != 0u) {  // warp-uniform: most steps improve nothing
        const unsigned mine = (im >> (h * GQ)) & GM;
        if (mine != 0u && g == 0) {
          atomicOr(pend_g + uq, mine);
          dirty_g[uq >> slog2] = 1u;
          improved += (uint32_t)__popc(mine);
          lanes_marked |= mine;
        }
        if (gbest_n != nullptr) {
          // smallest new value of the group, for the next round's window
          const uint32_t mn = __reduce_min_sync(kFull, imp ? nd[q] : kInf);
          if (mn != kInf && (threadIdx.x & 31) == 0) atomicMin(gbest_n, mn);
        }
      }
    }
  }
}

// The same step for groups of 64: lane l compares and lowers the pair of
// values of queries 2l and 2l + 1 (one 8-byte load of the target's line per
// arc for the warp's 256 bytes), and lane 0 marks the improved lanes of both
// halves in the 64-bit mask. sdv2 = the warp's [32][32] table of value pairs
// + l, or null with dv_own (a hub chunk); Dg_p = the group's state + 2l.
template <int QT>
__device__ __forceinline__ void g_step64(const GroupArgs &a, const uint4 *sarc, const uint2 *sdv2, uint2 dv_own,
                                         uint32_t *Dg_p, unsigned long long *pend_g, uint32_t *dirty_g, int lane,
                                         uint32_t &improved, bool chk) {
  const int slog2 = a.g.slog2;
#pragma unroll 1
  for (int j0 = 0; j0 < 32; j0 += kGUnroll64) {
    uint2 nd[kGUnroll64], cur[kGUnroll64];
    bool act0[kGUnroll64], act1[kGUnroll64];
#pragma unroll
    for (int q = 0; q < kGUnroll64; ++q) {
      const uint4 e = sarc[j0 + q];  // one broadcast read
      uint2 dv = make_uint2(kInf, kInf);
      if (e.z != kNoArc) dv = sdv2 != nullptr ? sdv2[e.z << 5] : dv_own;
      act0[q] = dv.x != kInf;
      act1[q] = dv.y != kInf;
      const uint32_t w = QT == Q_BFS ? 1u : e.y;
      uint32_t s0 = dv.x + w, s1 = dv.y + w;
      if (QT != Q_BFS && chk) {  // 2^32 - 1 reached: saturate and report
        if (act0[q] && (s0 < dv.x || s0 == kInf)) {
          atomicCAS(&a.ctrl->status, 0, (int)FG_ERR_OVERFLOW);
          s0 = kInf - 1u;
        }
        if (act1[q] && (s1 < dv.y || s1 == kInf)) {
          atomicCAS(&a.ctrl->status, 0, (int)FG_ERR_OVERFLOW);
          s1 = kInf - 1u;
        }
      }
      nd[q] = make_uint2(s0, s1);
      cur[q] = (act0[q] || act1[q]) ? *reinterpret_cast<const uint2 *>(Dg_p + ((size_t)e.x << 6)) : make_uint2(0u, 0u);
    }
#pragma unroll
    for (int q = 0; q < kGUnroll64; ++q) {
      const bool i0 = act0[q] && nd[q].x < cur[q].x, i1 = act1[q] && nd[q].y < cur[q].y;
      const uint32_t uq = sarc[j0 + q].x;  // read again rather than held in a register
      uint32_t *t = Dg_p + ((size_t)uq << 6);
      if (i0) atomicMin(t, nd[q].x);
      if (i1) atomicMin(t + 1, nd[q].y);
      const unsigned b0 = __ballot_sync(kFull, i0), b1 = __ballot_sync(kFull, i1);
      if ((b0 | b1) != 0u && lane == 0) {  // most steps improve nothing
        atomicOr(pend_g + uq, (unsigned long long)b0 | ((unsigned long long)b1 << 32));
        dirty_g[uq >> slog2] = 1u;
        improved += (uint32_t)(__popc(b0) + __popc(b1));
      }
    }
  }
}

template <int QT, int GQ>
__global__ void __launch_bounds__(kGThreads, 3) group_kernel(GroupArgs a) {
  extern __shared__ __align__(16) uint32_t g_smem[];
  __shared__ __align__(8) uint64_t s_full[2], s_empty[2], s_tma[2];
  __shared__ ItemDesc s_desc[2];
  // block counters (lane relaxations, improvements, arcs read, visits) and
  // block 0's phase clock, kept out of the registers of every thread
  __shared__ unsigned long long s_stat[4], s_ph[6], s_tprev;
  const int lane = lane_id(), wid = threadIdx.x >> 5;
  const bool producer = wid == kGCons;
  const DevGraph &G = a.g;
  const int S = G.S;
  constexpr int Gq = GQ;
  constexpr int LG = ilog2c(GQ);
  using M = typename GroupLanes<GQ>::M;  // pending-mask word of a vertex
  constexpr int SL = GroupLanes<GQ>::SL;  // arc slots per warp
  constexpr int MW = (int)sizeof(M) / 4;  // words per mask
  const int g = lane & (Gq - 1);    // query of the group held by this lane (G = 64: the pair)
  const int h = GQ == 64 ? 0 : lane >> LG;  // arc slot of this lane
  const size_t iw = group_item_words(S, Gq);
  M *const pend = reinterpret_cast<M *>(a.pend);
  // item buffer k: rp [S + 4], pm [S masks], vid [S]
  auto buf_rp = [&](uint32_t k) { return g_smem + k * iw; };
  auto buf_pm = [&](uint32_t k) { return reinterpret_cast<M *>(g_smem + k * iw + (S + 4)); };
  auto buf_vid = [&](uint32_t k) { return g_smem + k * iw + (S + 4) + MW * S; };
  // per consumer warp: the step's arcs (uint4[32]) and the batch's source values ([32][G])
  uint4 *sarc = reinterpret_cast<uint4 *>(g_smem + 2 * iw) + (size_t)(producer ? 0 : wid) * 32u;
  constexpr int kB = group_batch(GQ);  // listed vertices per consumer batch
  uint32_t *sdv = g_smem + 2 * iw + (size_t)kGCons * 128u + (size_t)(producer ? 0 : wid) * (size_t)kB * (uint32_t)Gq;
  Ctrl *c = a.ctrl;
  unsigned gen = *reinterpret_cast<volatile unsigned *>(&c->bar_gen);
  uint32_t it_base = 0;   // items this block has gone through (both buffers), the same in every warp
  uint32_t tma_bits = 0;  // producer: phase parity of s_tma[0] (bit 0) and s_tma[1] (bit 1)
  uint32_t r32 = 0, i32 = 0, a32 = 0;  // per-item counters, folded into s_stat after each item
#define FG_GPHASE(k)                                            \
  do {                                                          \
    if (blockIdx.x == 0 && threadIdx.x == 0) {                  \
      const uint64_t t_now = global_ns();                       \
      s_ph[k] += t_now - s_tprev;                               \
      s_tprev = t_now;                                          \
    }                                                           \
  } while (0)

  if (threadIdx.x == 0) {
    for (int k = 0; k < 4; ++k) s_stat[k] = 0ull;
    for (int k = 0; k < 6; ++k) s_ph[k] = 0ull;
    s_tprev = global_ns();
    for (int k = 0; k < 2; ++k) {
      mbar_init(&s_full[k], 1);
      mbar_init(&s_empty[k], kGCons);
      mbar_init(&s_tma[k], 1);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    fence_proxy_async_smem();
  }
  block_sync();

  const uint64_t K = (uint64_t)a.ngroups * (uint64_t)G.nparts;
  const uint64_t tid = (uint64_t)blockIdx.x * kGThreads + threadIdx.x, nthr = (uint64_t)gridDim.x * kGThreads;
  const size_t row = (size_t)a.npad;  // vertices per group row
  // values at or above ovf_lim can overflow when a weight is added
  const uint32_t ovf_lim = G.max_w >= kInf - 1u ? 0u : kInf - 1u - G.max_w;

  // ---- K0: state and masks (InitBuffers, first half); in serve mode only on
  //      the first launch on the state (later launches resume it) ----
  if (a.box == nullptr || a.init != 0u) {
    const uint64_t dwords = (uint64_t)a.ngroups * (uint64_t)a.npad * (uint64_t)Gq;
    for (uint64_t i = tid; i < dwords / 4u; i += nthr)
      reinterpret_cast<uint4 *>(a.D)[i] = make_uint4(kInf, kInf, kInf, kInf);
    const uint64_t pwords = 2ull * (uint64_t)a.ngroups * (uint64_t)a.npad * (uint64_t)MW;
    for (uint64_t i = tid; i < pwords / 4u; i += nthr) reinterpret_cast<uint4 *>(a.pend)[i] = make_uint4(0u, 0u, 0u, 0u);
    for (uint64_t i = tid; i < 2ull * K; i += nthr) a.dirty[i] = 0u;
    if (a.reach)
      for (uint64_t i = tid; i < (uint64_t)a.ngroups * (uint64_t)a.npad * (uint64_t)MW / 4u; i += nthr)
        reinterpret_cast<uint4 *>(a.reach)[i] = make_uint4(0u, 0u, 0u, 0u);
    if (a.gbest)
      for (uint64_t i = tid; i < 2ull * (uint64_t)a.ngroups; i += nthr) a.gbest[i] = kInf;
    if (a.gact)
      for (uint64_t i = tid; i < 2ull * (uint64_t)a.ngroups; i += nthr) a.gact[i] = 0u;
  }
  if (!grid_barrier(c, gen, a.watchdog_ns)) goto done;
  FG_GPHASE(0);

  // ---- INIT: each query's source gets value 0 and is pending in round 0
  //      (serve mode: sources come through the mailbox instead) ----
  for (uint64_t q = tid; a.box == nullptr && q < (uint64_t)a.nq; q += nthr) {
    const int32_t s = a.src[q];
    if (s < 0 || s >= G.n) {
      raise_status(c, FG_ERR_INVALID_ARG, kSiteSource);
      continue;
    }
    const uint32_t v = G.intl ? (uint32_t)G.intl[s] : (uint32_t)s;
    const uint32_t grp = (uint32_t)(q >> a.glog2), gq = (uint32_t)(q & (uint64_t)(Gq - 1));
    a.D[((size_t)grp * row + v) * (size_t)Gq + gq] = 0u;
    atomicOr(pend + (size_t)grp * row + v, group_bit<GQ>(gq));
    if (a.reach) atomicOr(reinterpret_cast<M *>(a.reach) + (size_t)grp * row + v, group_bit<GQ>(gq));
    a.dirty[(size_t)grp * G.nparts + (v >> G.slog2)] = 1u;
    if (a.gbest) atomicMin(a.gbest + grp, 0u);
  }
  if (!grid_barrier(c, gen, a.watchdog_ns)) goto done;
  FG_GPHASE(1);

  for (uint32_t round = a.round0;; ++round) {
    const uint32_t cur = round & 1u, nxt = cur ^ 1u;
    M *pend_c = pend + (size_t)cur * (size_t)a.ngroups * row;
    M *pend_n = pend + (size_t)nxt * (size_t)a.ngroups * row;
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
      if (a.gact)
        for (uint64_t i = tid; i < (uint64_t)a.ngroups; i += nthr) a.gact[(size_t)nxt * a.ngroups + i] = 0u;
      const uint64_t HK = (uint64_t)a.nhubs * (uint64_t)a.ngroups;
      for (uint64_t k = tid; k < HK; k += nthr) {
        const uint32_t grp = (uint32_t)(k / (uint64_t)a.nhubs), hi = (uint32_t)(k % (uint64_t)a.nhubs);
        const uint32_t v = a.hubs[hi];
        M *pw = pend_c + (size_t)grp * row + v;
        const M m = __ldcg(pw);
        if (m == 0u) continue;
        *pw = 0u;
        const uint32_t e0 = G.rp[v], e1 = G.rp[v + 1];
        const uint32_t nch = (e1 - e0 + a.hub_chunk - 1u) / a.hub_chunk;
        const uint32_t b = atomicAdd(&c->g_hub_items[cur], nch);
        for (uint32_t ch = 0; ch < nch && b + ch < a.hub_cap; ++ch) {
          a.items[b + ch] = make_uint4(grp, v, e0 + ch * a.hub_chunk, (uint32_t)m);
          if constexpr (GQ == 64) a.hub_hi[b + ch] = (uint32_t)(m >> 32);
        }
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
    if (GQ == 64 || a.box == nullptr) {
      if (n_hub + n_reg == 0u) break;
    } else if constexpr (GQ != 64) {
      // ---- serve mode: RETIRE lanes whose query has no pending work left, then
      //      ADMIT the mailbox's new requests into free lanes (next round) ----
      const uint32_t *gact_c = a.gact + (size_t)cur * a.ngroups;
      for (uint32_t grp = 0; grp < (uint32_t)a.ngroups; ++grp) {
        const uint32_t f = __ldcg(a.occ + grp) & ~__ldcg(gact_c + grp);  // the same in every block
        if (f == 0u) continue;
        uint32_t *Dg = a.D + (size_t)grp * row * (size_t)Gq;
        for (uint64_t v = tid; v < (uint64_t)G.n; v += nthr) {
          const uint64_t o = G.orig ? (uint64_t)G.orig[v] : v;
          if (a.reach) a.reach[(size_t)grp * row + v] &= ~f;  // BFS: the lanes have reached nothing
          uint32_t bits = f;
          while (bits != 0u) {
            const int gg = __ffs(bits) - 1;
            bits &= bits - 1u;
            uint32_t *pv = Dg + (v << LG) + (uint64_t)gg;
            a.res[((uint64_t)grp * (uint64_t)Gq + (uint64_t)gg) * (uint64_t)G.n + o] = __ldcg(pv);
            *pv = kInf;  // the lane starts over for its next request
          }
        }
      }
      if (!grid_barrier(c, gen, a.watchdog_ns)) goto done;
      if (blockIdx.x == 0 && wid == 0) {
        const uint32_t slots = (uint32_t)a.ngroups * (uint32_t)Gq;
        uint32_t admitted = 0;
        for (uint32_t sl = (uint32_t)lane; sl < slots; sl += 32u) {
          const uint32_t grp = sl >> LG, bit = 1u << (sl & (uint32_t)(Gq - 1));
          ServeSlot *bx = a.box->slot + sl;
          if ((__ldcg(a.occ + grp) & ~__ldcg(gact_c + grp) & bit) != 0u) {
            // the row is complete in res (written before the barrier): the
            // fence orders it and the status before the completion record
            st_volatile_sys(&bx->status, (int)FG_OK);
            __threadfence_system();
            st_volatile_sys(&bx->done_seq, a.seen[sl]);
            atomicAnd(a.occ + grp, ~bit);
          }
          if ((__ldcg(a.occ + grp) & bit) != 0u) continue;
          const uint32_t seq = ld_volatile_sys(&bx->seq);
          if (seq == a.seen[sl]) continue;
          fence_acq_rel_sys();
          const int32_t src = (int32_t)ld_volatile_sys(reinterpret_cast<uint32_t *>(&bx->src));
          a.seen[sl] = seq;
          st_volatile_sys(&bx->ack, seq);
          if (src < 0 || src >= G.n) {  // rejected at once: the row is not written
            st_volatile_sys(&bx->status, (int)FG_ERR_INVALID_ARG);
            __threadfence_system();
            st_volatile_sys(&bx->done_seq, seq);
            continue;
          }
          const uint32_t v = G.intl ? (uint32_t)G.intl[src] : (uint32_t)src;
          a.D[((size_t)grp * row + v) * (size_t)Gq + (sl & (uint32_t)(Gq - 1))] = 0u;
          atomicOr(pend_n + (size_t)grp * row + v, bit);
          dirty_n[(size_t)grp * G.nparts + (v >> G.slog2)] = 1u;
          atomicOr(a.gact + (size_t)nxt * a.ngroups + grp, bit);
          atomicOr(a.occ + grp, bit);
          if (a.gbest) atomicMin(a.gbest + (size_t)nxt * a.ngroups + grp, 0u);
          if (a.reach) {  // BFS: the source is reached; levels count from the next round
            atomicOr(a.reach + (size_t)grp * row + v, bit);
            a.lstart[sl] = round + 1u;
          }
          ++admitted;
        }
        __syncwarp();
        uint32_t busy = 0;
        for (uint32_t grp = (uint32_t)lane; grp < (uint32_t)a.ngroups; grp += 32u) busy |= __ldcg(a.occ + grp);
        busy = __reduce_or_sync(kFull, busy);
        admitted = __reduce_add_sync(kFull, admitted);
        // idle (nothing to process, no lane held) or told to stop: the launch
        // ends; the host relaunches it when a request waits unacknowledged
        const bool stop = ld_volatile_sys(&a.box->stop) != 0u;
        if (lane == 0) c->g_exit = (stop || (n_hub + n_reg == 0u && busy == 0u && admitted == 0u)) ? 1u : 0u;
      }
    }
    if (a.box == nullptr && round >= a.max_rounds) {
      if (threadIdx.x == 0) raise_status(c, FG_ERR_TIMEOUT, kSiteRounds);
      break;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      c->rounds += 1ull;
      if ((unsigned long long)n_hub + n_reg > c->max_round_ops) c->max_round_ops = (unsigned long long)n_hub + n_reg;
    }
    // ---- PROCESS ----
    if (producer) {
      // -- claim, stage, list, publish; every wait is bounded --
      uint32_t it = it_base;
      for (;;) {
        const uint32_t k = it & 1u, use = it >> 1;
        // every wait's outcome is made warp-uniform before anyone acts on it
        if (use > 0u && !__all_sync(kFull, mbar_wait(&s_empty[k], (use - 1u) & 1u, a.watchdog_ns))) {
          if (lane == 0) raise_status(c, FG_ERR_TIMEOUT, kSiteStage);
          break;  // the consumers time out on their own waits
        }
        uint32_t idx = 0;
        if (lane == 0) {
          idx = atomicAdd(&c->g_next[cur], 1u);
          if (ld_volatile_i32(&c->abort)) idx = n_hub + n_reg;
        }
        idx = __shfl_sync(kFull, idx, 0);
        ItemDesc d{kItemEnd, 0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u, 0ull};
        if (idx < n_hub) {
          const uint4 itm = __ldcg(a.items + idx);
          const uint32_t e1 = G.rp[itm.y + 1];
          d.kind = kItemHub;
          d.grp = itm.x;
          d.pv = itm.y;
          d.eb = itm.z;
          d.ee = itm.z + a.hub_chunk < e1 ? itm.z + a.hub_chunk : e1;
          d.m = itm.w;
          if constexpr (GQ == 64) d.m |= (unsigned long long)__ldcg(a.hub_hi + idx) << 32;
          d.n = (d.ee - d.eb + 31u) / 32u;
        } else if (idx < n_hub + n_reg) {
          const uint32_t key = __ldcg(a.items + a.hub_cap + (idx - n_hub)).x;
          const uint32_t grp = key / (uint32_t)G.nparts, p = key - grp * (uint32_t)G.nparts;
          const uint32_t base = p << G.slog2;
          M *pm_g = pend_c + (size_t)grp * row + base;
          uint32_t *rp_s = buf_rp(k), *vid_s = buf_vid(k);
          M *pm_s = buf_pm(k);
          // stage the row offsets and the group's pending masks (one bulk
          // phase; the expected bytes are announced before the copies); the
          // buffer's previous readers are done (empty barrier), so the proxy
          // fence orders their reads before the bulk writes
          if (lane == 0) {
            const uint32_t b_rp = (uint32_t)(S + 4) * 4u, b_pm = (uint32_t)S * (uint32_t)sizeof(M);
            fence_proxy_async_smem();
            mbar_arrive_expect_tx(&s_tma[k], b_rp + b_pm);
            bulk_g2s(rp_s, G.rp + base, b_rp, &s_tma[k]);
            bulk_g2s(pm_s, pm_g, b_pm, &s_tma[k]);
          }
          const uint32_t par = (tma_bits >> k) & 1u;
          const bool ok = __all_sync(kFull, mbar_wait(&s_tma[k], par, a.watchdog_ns));
          if (!ok) {
            if (lane == 0) {
              raise_status(c, FG_ERR_TIMEOUT, kSiteStage);
              (void)mbar_wait(&s_tma[k], par, 1000000ull);  // the copies in flight, once more, bounded
            }
            break;
          }
          tma_bits ^= 1u << k;
          if (a.check_staging) {
            // self-test: the landed words equal global memory (row offsets
            // never change; this round's masks change only when cleared below)
            bool bad = false;
            for (int i = lane; i < S + 4; i += 32) bad |= rp_s[i] != __ldg(G.rp + base + i);
            for (int i = lane; i < S; i += 32) bad |= pm_s[i] != __ldcg(pm_g + i);
            if (__any_sync(kFull, bad) && lane == 0) raise_status(c, FG_ERR_CUDA, kSiteStageCheck);
          }
          // this round's masks of the item are taken: clear them for reuse
          for (int i = lane; i < ((S * MW) >> 2); i += 32)
            reinterpret_cast<uint4 *>(pm_g)[i] = make_uint4(0u, 0u, 0u, 0u);
          // list the pending vertices with an arc: those with many pending
          // lanes from the front of vid, the sparse ones (no window only)
          // from its back
          uint32_t cnt = 0, cnt_s = 0;
          const bool use_sparse = QT != Q_BFS && GQ >= 32 && a.window == 0u;
          const unsigned lt = (1u << lane) - 1u;
          for (int i0 = 0; i0 < S; i0 += 32) {
            const int i = i0 + lane;
            const uint32_t deg = rp_s[i + 1] - rp_s[i];
            const M mk = pm_s[i];
            const bool keep = mk != 0u && deg > 0u;
            int pc;
            if constexpr (GQ == 64) pc = __popcll(mk);
            else pc = __popc(mk);
            const bool sp = keep && use_sparse && pc <= kSparseT;
            const unsigned bd = __ballot_sync(kFull, keep && !sp), bs = __ballot_sync(kFull, sp);
            if (keep && !sp) vid_s[cnt + (uint32_t)__popc(bd & lt)] = (uint32_t)i;
            if (sp) vid_s[S - 1 - (cnt_s + (uint32_t)__popc(bs & lt))] = (uint32_t)i;
            cnt += (uint32_t)__popc(bd);
            cnt_s += (uint32_t)__popc(bs);
          }
          d.kind = kItemPart;
          d.grp = grp;
          d.pv = p;
          d.n = cnt;
          d.ns = cnt_s;
        }
        if (lane == 0) {
          s_desc[k] = d;
          if (d.kind != kItemEnd) s_stat[3] += 1ull;  // the producer's lane 0 alone counts visits
        }
        __syncwarp();  // every lane's list writes precede the publishing arrival
        if (lane == 0) mbar_arrive(&s_full[k]);
        ++it;
        if (d.kind == kItemEnd) break;
      }
      it_base = it;
    } else {
      // -- consumers: batches of the published items, in order --
      uint32_t it = it_base;
      for (;;) {
        const uint32_t k = it & 1u, use = it >> 1;
        if (!__all_sync(kFull, mbar_wait(&s_full[k], use & 1u, a.watchdog_ns))) {
          if (lane == 0) raise_status(c, FG_ERR_TIMEOUT, kSiteStage);
          break;
        }
        const ItemDesc d = s_desc[k];
        ++it;
        if (d.kind == kItemEnd) {
          __syncwarp();
          if (lane == 0) mbar_arrive(&s_empty[k]);
          break;
        }
        uint32_t *Dg = a.D + (size_t)d.grp * row * (size_t)Gq;
        uint32_t *Dg_g = Dg + (GQ == 64 ? 2 * lane : g);  // this lane's value (G = 64: pair) of vertex 0
        uint32_t gacc = 0u;  // lanes this warp marked pending for the next round (serve mode)
        M *pend_g = pend_n + (size_t)d.grp * row;
        uint32_t *dirty_g = dirty_n + (size_t)d.grp * G.nparts;
        uint32_t *gb_n = a.gbest ? a.gbest + (size_t)nxt * a.ngroups + d.grp : nullptr;
        // Steps of 32 arcs, lane l holding arc l. Two steps ahead of the one
        // being relaxed, a lane loads its arc (target, weight); one step ahead,
        // it asks L2 for the arc's target line (prefetch.global.L2), so the
        // relaxation's loads of target values find their lines on chip
        // without holding registers while they travel.
        auto run = [&](uint32_t nsteps, auto make, auto sdv_g, auto dv_own, bool chk) {
          const uint4 none = make_uint4(0u, 1u, kNoArc, 0u);
          uint4 a0 = make(0u);
          uint4 a1 = nsteps > 1u ? make(1u) : none;
          // a vertex's line of the group: 32-256 bytes (two 128-byte lines for G = 64)
          auto prefetch_line = [&](uint32_t v) {
            const uint32_t *p = Dg + ((size_t)v << LG);
            prefetch_l2(p);
            if constexpr (GQ == 64) prefetch_l2(p + 32);
          };
          if (a0.z != kNoArc) prefetch_line(a0.x);
          for (uint32_t i = 0; i < nsteps; ++i) {
            sarc[lane] = a0;
            __syncwarp();
            if (a1.z != kNoArc) prefetch_line(a1.x);
            const uint4 a2 = i + 2u < nsteps ? make(i + 2u) : none;
            if constexpr (GQ == 64)
              g_step64<QT>(a, sarc, sdv_g, dv_own, Dg_g, pend_g, dirty_g, lane, i32, chk);
            else
              g_step<QT, GQ>(a, sarc, sdv_g, dv_own, Dg_g, pend_g, dirty_g, gb_n, g, h, i32, gacc, chk);
            __syncwarp();  // sarc is rewritten by the next step
            a0 = a1;
            a1 = a2;
          }
        };
        if constexpr (QT == Q_BFS) {
          // BFS: rounds are levels, so a query's level of a vertex is fixed
          // when the query first reaches it. reach[v] holds the queries that
          // have reached v. A lane takes one arc at a time and sets the
          // frontier lanes F of the arc's source that are new in the
          // target's reach; only those lanes are marked pending and get
          // their level. One 4- or 8-byte word per arc replaces the
          // target's line.
          M *reach_g = reinterpret_cast<M *>(a.reach) + (size_t)d.grp * row;
          const int slog2 = G.slog2;
          const uint32_t lvl = round + 1u;  // the level reached in this round (serve mode: minus the lane's start)
          constexpr int kU = 4;  // arcs per lane with their loads in flight at once
          // relax up to kU arcs per lane: targets v[u] (kNoArc: none) from frontiers F[u]
          auto visit = [&](const uint32_t *v, const M *F) {
            M nw[kU];
#pragma unroll
            for (int u = 0; u < kU; ++u) nw[u] = v[u] != kNoArc ? (F[u] & ~reach_g[v[u]]) : (M)0u;
#pragma unroll
            for (int u = 0; u < kU; ++u) {
              if (nw[u] == 0u) continue;
              M fresh = nw[u] & ~atomicOr(reach_g + v[u], nw[u]);
              if (fresh == 0u) continue;
              atomicOr(pend_g + v[u], fresh);
              dirty_g[v[u] >> slog2] = 1u;
              if constexpr (GQ == 64) i32 += (uint32_t)__popcll(fresh);
              else {
                i32 += (uint32_t)__popc(fresh);
                gacc |= fresh;
              }
              uint32_t *Dv = Dg + ((size_t)v[u] << LG);
              while (fresh != 0u) {
                int bp;
                if constexpr (GQ == 64) bp = __ffsll((long long)fresh) - 1;
                else bp = __ffs(fresh) - 1;
                fresh &= fresh - 1u;
                const uint32_t gq =
                    GQ == 64 ? ((((uint32_t)bp & 31u) << 1) | ((uint32_t)bp >> 5)) : (uint32_t)bp;
                Dv[gq] = a.lstart ? lvl - a.lstart[(size_t)d.grp * Gq + gq] : lvl;
              }
            }
          };
          if (d.kind == kItemHub) {
            const M F = (M)d.m;
            uint32_t fpc;
            if constexpr (GQ == 64) fpc = (uint32_t)__popcll(F);
            else fpc = (uint32_t)__popc(F);
            for (;;) {
              uint32_t s0 = 0;
              if (lane == 0) s0 = atomicAdd(&s_desc[k].next, 4u);  // four steps of 32 arcs at a time
              s0 = __shfl_sync(kFull, s0, 0);
              if (s0 >= d.n) break;
              uint32_t v[kU];
              M Fs[kU];
#pragma unroll
              for (int u = 0; u < kU; ++u) {
                const uint32_t e = d.eb + (s0 + (uint32_t)u) * 32u + (uint32_t)lane;
                const bool has = s0 + (uint32_t)u < d.n && e < d.ee;
                v[u] = has ? __ldg(G.adj + e) : kNoArc;
                Fs[u] = F;
                a32 += has ? 1u : 0u;
                r32 += has ? fpc : 0u;
              }
              visit(v, Fs);
            }
          } else {
            const uint32_t base = d.pv << G.slog2;
            const uint32_t *rp_s = buf_rp(k), *vid_s = buf_vid(k);
            const M *pm_s = buf_pm(k);
            (void)base;
            for (;;) {
              uint32_t b0 = 0;
              if (lane == 0) b0 = atomicAdd(&s_desc[k].next, 32u);
              b0 = __shfl_sync(kFull, b0, 0);
              if (b0 >= d.n) break;
              const uint32_t j = b0 + (uint32_t)lane;
              const bool valid = j < d.n;
              const uint32_t li = valid ? vid_s[j] : 0u;
              const M m = valid ? pm_s[li] : (M)0u;
              const uint32_t a0 = valid ? rp_s[li] : 0u;
              const uint32_t deg = valid ? rp_s[li + 1] - a0 : 0u;
              if constexpr (GQ == 64) r32 += deg * (uint32_t)__popcll(m);
              else r32 += deg * (uint32_t)__popc(m);
              const uint32_t incl = warp_incl_scan(deg);
              const uint32_t exd = incl - deg;
              const uint32_t tot = __shfl_sync(kFull, incl, 31);
              for (uint32_t t0 = 0; t0 < tot; t0 += 32u * kU) {
                uint32_t v[kU];
                M Fs[kU];
#pragma unroll
                for (int u = 0; u < kU; ++u) {
                  const uint32_t t = t0 + (uint32_t)u * 32u + (uint32_t)lane;
                  const bool has = t < tot;
                  const int L = owner_lane(exd, has ? t : 0u);
                  const uint32_t eL = __shfl_sync(kFull, a0, L) + (t - __shfl_sync(kFull, exd, L));
                  const M FL = __shfl_sync(kFull, m, L);
                  v[u] = has ? __ldg(G.adj + eL) : kNoArc;
                  Fs[u] = FL;
                  a32 += has ? 1u : 0u;
                }
                visit(v, Fs);
              }
            }
          }
        } else if (d.kind == kItemHub) {
          // this lane's value(s) of the hub, kInf where not pending
          using V = std::conditional_t<GQ == 64, uint2, uint32_t>;
          V dv;
          uint32_t nact;  // values of this lane that relax the chunk
          bool near;      // a sum can reach 2^32 - 1 only from a value within max_w of it
          if constexpr (GQ == 64) {
            const bool p0 = ((d.m >> lane) & 1ull) != 0ull, p1 = ((d.m >> (32 + lane)) & 1ull) != 0ull;
            dv = make_uint2(kInf, kInf);
            if (p0 || p1) {
              const uint2 t = __ldcg(reinterpret_cast<const uint2 *>(Dg_g + ((size_t)d.pv << LG)));
              if (p0) dv.x = t.x;
              if (p1) dv.y = t.y;
            }
            nact = (dv.x != kInf ? 1u : 0u) + (dv.y != kInf ? 1u : 0u);
            near = (dv.x != kInf && dv.x >= ovf_lim) || (dv.y != kInf && dv.y >= ovf_lim);
          } else {
            dv = kInf;
            if (((d.m >> g) & 1ull) != 0ull) dv = __ldcg(Dg_g + ((size_t)d.pv << LG));
            nact = dv != kInf ? 1u : 0u;
            near = dv != kInf && dv >= ovf_lim;
          }
          const bool chk_hub = __any_sync(kFull, near);
          for (;;) {
            uint32_t s0 = 0;
            if (lane == 0) s0 = atomicAdd(&s_desc[k].next, 4u);  // four steps of 32 arcs at a time
            s0 = __shfl_sync(kFull, s0, 0);
            if (s0 >= d.n) break;
            const uint32_t ns = d.n - s0 < 4u ? d.n - s0 : 4u;
            if (nact != 0u) {  // this lane relaxes every arc of the claimed steps
              const uint32_t e_lo = d.eb + s0 * 32u, e_hi = d.eb + (s0 + ns) * 32u;
              r32 += nact * ((e_hi < d.ee ? e_hi : d.ee) - e_lo);
            }
            auto make = [&](uint32_t i) {
              const uint32_t e = d.eb + (s0 + i) * 32u + (uint32_t)lane;
              const bool has = e < d.ee;
              a32 += has ? 1u : 0u;
              return make_uint4(has ? __ldg(G.adj + e) : 0u,
                                (has && QT != Q_BFS && G.wt != nullptr) ? __ldg(G.wt + e) : 1u,
                                has ? 0u : kNoArc, 0u);
            };
            run(ns, make, static_cast<const V *>(nullptr), dv, chk_hub);
          }
        } else {
          const uint32_t base = d.pv << G.slog2;
          const uint32_t *rp_s = buf_rp(k), *vid_s = buf_vid(k);
          const M *pm_s = buf_pm(k);
          const uint32_t bound =
              (a.window != 0u && a.gbest != nullptr)
                  ? sat_add_u32(__ldcg(a.gbest + (size_t)cur * a.ngroups + d.grp), a.window)
                  : kInf;
          for (;;) {
            uint32_t b0 = 0;
            if (lane == 0) b0 = atomicAdd(&s_desc[k].next, (uint32_t)kB);
            b0 = __shfl_sync(kFull, b0, 0);
            if (b0 >= d.n) break;
            const uint32_t j = b0 + (uint32_t)lane;
            const bool valid = lane < kB && j < d.n;
            const uint32_t li = valid ? vid_s[j] : 0u;
            const M m = valid ? pm_s[li] : (M)0u;
            const uint32_t a0 = valid ? rp_s[li] : 0u;
            const uint32_t deg = valid ? rp_s[li + 1] - a0 : 0u;
            const uint32_t incl = warp_incl_scan(deg);
            const uint32_t exd = incl - deg;
            const uint32_t tot = __shfl_sync(kFull, incl, 31);
            // the batch's source values, fresh from L2 (the pending bit was set
            // because the value fell; an older copy could miss that fall): row
            // L of sdv holds vertex L's values of the group, kInf where not
            // pending. Under a window, values at or beyond the group's bound
            // stay pending for a later round (Delta-stepping across rounds).
            bool big = false;  // some source value within max_w of 2^32 - 1 (sums need the check)
            if constexpr (GQ == 64) {
              // pairs: row L of the [16][32] pair table, lane l = queries 2l, 2l + 1
              uint2 *sdv2 = reinterpret_cast<uint2 *>(sdv);
#pragma unroll 4
              for (int L = 0; L < kB; ++L) {
                const uint32_t vL = __shfl_sync(kFull, li, L);
                const M mL = __shfl_sync(kFull, m, L);
                const bool p0 = ((mL >> lane) & 1ull) != 0ull, p1 = ((mL >> (32 + lane)) & 1ull) != 0ull;
                uint2 dd = make_uint2(kInf, kInf);
                if (p0 || p1) {
                  const uint2 t = __ldcg(reinterpret_cast<const uint2 *>(Dg_g + ((size_t)(base + vL) << LG)));
                  if (p0) dd.x = t.x;
                  if (p1) dd.y = t.y;
                }
                sdv2[(L << 5) + lane] = dd;
                big |= (dd.x != kInf && dd.x >= ovf_lim) || (dd.y != kInf && dd.y >= ovf_lim);
                const uint32_t degL = __shfl_sync(kFull, deg, L);
                r32 += degL * ((dd.x != kInf ? 1u : 0u) + (dd.y != kInf ? 1u : 0u));
              }
            } else {
#pragma unroll 4
            for (int L0 = 0; L0 < 32; L0 += SL) {
              const int L = L0 + h;
              const uint32_t vL = __shfl_sync(kFull, li, L);
              const uint32_t mL = __shfl_sync(kFull, m, L);
              uint32_t dd = kInf;
              if (((mL >> g) & 1u) != 0u) dd = __ldcg(Dg_g + ((size_t)(base + vL) << LG));
              if (bound != kInf) {  // block-uniform
                const bool def = dd != kInf && dd >= bound;
                const unsigned dm = __ballot_sync(kFull, def);
                const unsigned mine = (dm >> (h * Gq)) & (Gq == 32 ? 0xFFFFFFFFu : ((1u << Gq) - 1u));
                if (mine != 0u && g == 0) {
                  atomicOr(pend_g + base + vL, mine);
                  dirty_g[d.pv] = 1u;
                  gacc |= mine;
                }
                if (gb_n != nullptr) {
                  const uint32_t mn = __reduce_min_sync(kFull, def ? dd : kInf);
                  if (mn != kInf && lane == 0) atomicMin(gb_n, mn);
                }
                if (def) dd = kInf;
              }
              sdv[(L << LG) + g] = dd;
              big |= dd != kInf && dd >= ovf_lim;
              const uint32_t degL = __shfl_sync(kFull, deg, L);
              if (dd != kInf) r32 += degL;  // this lane relaxes every arc of vertex L
            }
            }
            __syncwarp();
            auto make = [&](uint32_t i) {
              const uint32_t t = i * 32u + (uint32_t)lane;
              const bool has = t < tot;
              const int L = owner_lane(exd, has ? t : 0u);
              const uint32_t eL = __shfl_sync(kFull, a0, L) + (t - __shfl_sync(kFull, exd, L));
              a32 += has ? 1u : 0u;
              return make_uint4(has ? __ldg(G.adj + eL) : 0u,
                                (has && QT != Q_BFS && G.wt != nullptr) ? __ldg(G.wt + eL) : 1u,
                                has ? (uint32_t)L : kNoArc, 0u);
            };
            if constexpr (GQ == 64)
              run((tot + 31u) / 32u, make, static_cast<const uint2 *>(reinterpret_cast<uint2 *>(sdv) + lane),
                  make_uint2(kInf, kInf), __any_sync(kFull, big));
            else
              run((tot + 31u) / 32u, make, static_cast<const uint32_t *>(sdv + g), kInf, __any_sync(kFull, big));
            __syncwarp();  // sdv is rewritten by the next batch
          }
          if constexpr (GQ >= 32) {
            // the sparse vertices, 32 at a time: lanes take (arc, pending
            // query) pairs, kSparseT slots per arc, and each pair reads and
            // lowers one 4-byte value of its target
            constexpr uint32_t kT = kSparseT, kAPS = 32 / kSparseT;  // slots per arc, arcs per step
            uint32_t *sval = sdv;              // [32][kT] source values of the batch's vertices
            uint32_t *sgq = sdv + 32u * kT;    // [32][kT] their queries
            const int slog2 = G.slog2;
            for (;;) {
              uint32_t b0 = 0;
              if (lane == 0) b0 = atomicAdd(&s_desc[k].next_s, 32u);
              b0 = __shfl_sync(kFull, b0, 0);
              if (b0 >= d.ns) break;
              const uint32_t j = b0 + (uint32_t)lane;
              const bool valid = j < d.ns;
              const uint32_t li = valid ? vid_s[S - 1 - j] : 0u;
              M mk = valid ? pm_s[li] : (M)0u;
              const uint32_t a0 = valid ? rp_s[li] : 0u;
              const uint32_t deg = valid ? rp_s[li + 1] - a0 : 0u;
              // this lane's vertex: the values of its pending queries, in bit
              // order (fresh from L2, as for the dense batches)
              const uint32_t *Dv = Dg + ((size_t)(base + li) << LG);
              uint32_t pc = 0;
              bool near = false;
              while (mk != 0u) {
                int bp;
                if constexpr (GQ == 64) bp = __ffsll((long long)mk) - 1;
                else bp = __ffs(mk) - 1;
                mk &= mk - 1u;
                const uint32_t gq =
                    GQ == 64 ? ((((uint32_t)bp & 31u) << 1) | ((uint32_t)bp >> 5)) : (uint32_t)bp;
                const uint32_t dv = __ldcg(Dv + gq);
                sval[lane * kT + pc] = dv;
                sgq[lane * kT + pc] = gq;
                near |= dv != kInf && dv >= ovf_lim;
                ++pc;
              }
              r32 += deg * pc;  // this lane's vertex relaxes every arc for each pending query
              const bool chk_s = __any_sync(kFull, near);
              const uint32_t incl = warp_incl_scan(deg);
              const uint32_t exd = incl - deg;
              const uint32_t tot = __shfl_sync(kFull, incl, 31);
              __syncwarp();
              constexpr int kU = 4;  // steps with their loads in flight at once
              for (uint32_t t0 = 0; t0 < tot; t0 += kAPS * kU) {
                uint32_t nd[kU], cv[kU], gq[kU], vv[kU];
                bool on[kU];
#pragma unroll
                for (int u = 0; u < kU; ++u) {
                  const uint32_t t = t0 + u * kAPS + (uint32_t)lane / kT, slot = (uint32_t)lane % kT;
                  const bool has = t < tot;
                  const int L = owner_lane(exd, has ? t : 0u);
                  const uint32_t pcL = __shfl_sync(kFull, pc, L);
                  const uint32_t eL = __shfl_sync(kFull, a0, L) + (t - __shfl_sync(kFull, exd, L));
                  a32 += (has && slot == 0u) ? 1u : 0u;  // the arc is read once, counted by its first slot
                  on[u] = has && slot < pcL;
                  nd[u] = kInf;
                  cv[u] = 0u;
                  gq[u] = 0u;
                  vv[u] = 0u;
                  if (on[u]) {
                    const uint32_t v = __ldg(G.adj + eL);
                    const uint32_t w = (QT != Q_BFS && G.wt != nullptr) ? __ldg(G.wt + eL) : 1u;
                    const uint32_t dv = sval[L * kT + slot];
                    gq[u] = sgq[L * kT + slot];
                    uint32_t x = dv + w;
                    if (QT != Q_BFS && chk_s && (x < dv || x == kInf)) {  // 2^32 - 1 reached
                      atomicCAS(&c->status, 0, (int)FG_ERR_OVERFLOW);
                      x = kInf - 1u;
                    }
                    nd[u] = x;
                    vv[u] = v;
                    cv[u] = Dg[((size_t)v << LG) + gq[u]];
                  }
                }
#pragma unroll
                for (int u = 0; u < kU; ++u) {
                  if (on[u] && nd[u] < cv[u]) {  // a stale value is an upper bound, as in the dense step
                    atomicMin(Dg + ((size_t)vv[u] << LG) + gq[u], nd[u]);
                    atomicOr(pend_g + vv[u], group_bit<GQ>(gq[u]));
                    dirty_g[vv[u] >> slog2] = 1u;
                    ++i32;
                    if constexpr (GQ != 64) gacc |= (uint32_t)group_bit<GQ>(gq[u]);
                  }
                }
              }
              __syncwarp();  // sval and sgq are rewritten by the next batch
            }
          }
        }
        {
          const unsigned long long r = warp_sum((unsigned long long)r32), im = warp_sum((unsigned long long)i32),
                                   ar = warp_sum((unsigned long long)a32);
          if (lane == 0) {
            atomicAdd(&s_stat[0], r);
            atomicAdd(&s_stat[1], im);
            atomicAdd(&s_stat[2], ar);
          }
        }
        r32 = 0u;
        i32 = 0u;
        a32 = 0u;
        if (GQ != 64 && a.gact != nullptr) {
          gacc = __reduce_or_sync(kFull, gacc);
          if (lane == 0 && gacc != 0u) atomicOr(a.gact + (size_t)nxt * a.ngroups + d.grp, gacc);
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&s_empty[k]);  // this warp is done with buffer k
      }
      it_base = it;
    }
    if (!grid_barrier(c, gen, a.watchdog_ns)) goto done;
    FG_GPHASE(5);
    // serve mode: leave when idle or told to stop, or yield after max_rounds
    // rounds with the state intact (the next launch resumes at round + 1)
    if (a.box != nullptr &&
        (*reinterpret_cast<volatile unsigned *>(&c->g_exit) != 0u || round + 1u - a.round0 >= a.max_rounds))
      break;
  }
done:
#undef FG_GPHASE
  block_sync();  // every warp has folded its counters
  if (threadIdx.x == 0) {
    if (blockIdx.x == 0) {
      s_ph[2] += global_ns() - s_tprev;
      for (int k = 0; k < 6; ++k) atomicAdd(&c->phase_ns[k], s_ph[k]);
    }
    atomicAdd(&c->edges, s_stat[0]);
    atomicAdd(&c->ops, s_stat[1]);
    atomicAdd(&c->arcs_read, s_stat[2]);
    atomicAdd(&c->visits, s_stat[3]);
  }
}

// D[group][v][g] (internal order) -> out[row(group * G + g)][orig(v)] for v < n,
// row(j) = rowmap[j] (or j without a map). A block moves 32 vertices of one
// group: 32 * G words read as whole lines, transposed in shared memory,
// written as G runs of 32 values.
__global__ void __launch_bounds__(256) group_out_kernel(const uint32_t *D, uint32_t *out, const int32_t *orig,
                                                        const int32_t *rowmap, int64_t n, int64_t npad, int32_t G,
                                                        int32_t glog2, int32_t nq, int64_t tiles_per_group) {
  __shared__ uint32_t t[64][33];
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
      const int64_t r = rowmap ? (int64_t)rowmap[q] : q;
      out[r * n + o] = t[gq][vl];
    }
  }
}

// Key of each query's source for its place in the batch: the sum of its
// out-neighbours' degrees (two-hop reach), or, by_place, its internal id
// counted down (queries from nearby sources side by side: partitions that
// keep most arcs inside hold nearby vertices under consecutive ids). One warp
// per query; an out-of-range source gets 0 and is reported by the engine's
// INIT.
__global__ void __launch_bounds__(256) group_key_kernel(DevGraph G, const int32_t *src, int32_t nq,
                                                        unsigned long long *key, int by_place) {
  const int64_t q = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (q >= nq) return;
  const int32_t s = src[q];
  unsigned long long sum = 0;
  if (s >= 0 && s < G.n && by_place) {
    if (lane == 0) key[q] = (unsigned long long)(uint32_t)G.n - (G.intl ? (uint32_t)G.intl[s] : (uint32_t)s);
    return;
  }
  if (s >= 0 && s < G.n) {
    const uint32_t v = G.intl ? (uint32_t)G.intl[s] : (uint32_t)s;
    const uint32_t e0 = G.rp[v], e1 = G.rp[v + 1];
    for (uint32_t e = e0 + (uint32_t)lane; e < e1; e += 32u) {
      const uint32_t u = G.adj[e];
      sum += (unsigned long long)(G.rp[u + 1] - G.rp[u]);
    }
  }
  for (int o = 16; o > 0; o >>= 1) sum += __shfl_down_sync(0xFFFFFFFFu, sum, o);
  if (lane == 0) key[q] = sum;
}

// Slot of each query: the number of queries with a larger key, or the same key
// and a smaller index (a stable descending order). Keys are read in tiles of
// 1,024 through shared memory.
__global__ void __launch_bounds__(256) group_rank_kernel(const unsigned long long *key, const int32_t *src,
                                                         int32_t nq, int32_t *perm, int32_t *psrc) {
  __shared__ unsigned long long tk[1024];
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const unsigned long long kq = q < nq ? key[q] : 0ull;
  int64_t rank = 0;
  for (int64_t t0 = 0; t0 < nq; t0 += 1024) {
    const int64_t cnt = nq - t0 < 1024 ? nq - t0 : 1024;
    __syncthreads();
    for (int64_t i = threadIdx.x; i < cnt; i += blockDim.x) tk[i] = key[t0 + i];
    __syncthreads();
    if (q < nq)
      for (int64_t i = 0; i < cnt; ++i) {
        const unsigned long long k = tk[i];
        rank += (k > kq || (k == kq && t0 + i < q)) ? 1 : 0;
      }
  }
  if (q < nq) {
    perm[rank] = (int32_t)q;
    psrc[rank] = src[q];
  }
}

static const void *group_fn(int qtype, int G) {
  if (qtype == Q_BFS) {
    if (G == 8) return (const void *)group_kernel<Q_BFS, 8>;
    if (G == 16) return (const void *)group_kernel<Q_BFS, 16>;
    if (G == 64) return (const void *)group_kernel<Q_BFS, 64>;
    return (const void *)group_kernel<Q_BFS, 32>;
  }
  if (G == 8) return (const void *)group_kernel<Q_SSSP, 8>;
  if (G == 16) return (const void *)group_kernel<Q_SSSP, 16>;
  if (G == 64) return (const void *)group_kernel<Q_SSSP, 64>;
  return (const void *)group_kernel<Q_SSSP, 32>;
}

bool group_fits(int S, int G) {
  int dev = 0, optin = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return false;
  if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) return false;
  return group_smem_bytes(S, G) <= (size_t)optin;
}

cudaError_t group_grid_size(int S, int G, int *blocks, int *threads, size_t *smem) {
  *threads = kGThreads;
  *smem = group_smem_bytes(S, G);
  int best = 1 << 30, dev = 0, sms = 0;
  cudaError_t e;
  for (int qt = 0; qt < 2; ++qt) {
    const void *fn = group_fn(qt, G);
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
  return cudaLaunchCooperativeKernel(group_fn(a.qtype, a.G), dim3(blocks), dim3(threads), args, smem, s);
}

cudaError_t launch_group_out(const GroupArgs &a, uint32_t *out, const int32_t *rowmap, cudaStream_t s) {
  const int64_t n = a.g.n;
  const int64_t tiles = (n + 31) / 32;
  const int64_t grid = tiles * (int64_t)a.ngroups;
  if (grid <= 0) return cudaSuccess;
  group_out_kernel<<<(unsigned)grid, 256, 0, s>>>(a.D, out, a.g.orig, rowmap, n, a.npad, a.G, a.glog2, a.nq, tiles);
  return cudaGetLastError();
}

cudaError_t launch_group_order(const DevGraph &g, const int32_t *src, int32_t nq, bool by_place,
                               unsigned long long *key, int32_t *perm, int32_t *psrc, cudaStream_t s) {
  if (nq <= 0) return cudaSuccess;
  const int64_t warps_grid = ((int64_t)nq * 32 + 255) / 256;
  group_key_kernel<<<(unsigned)warps_grid, 256, 0, s>>>(g, src, nq, key, by_place ? 1 : 0);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  group_rank_kernel<<<(unsigned)((nq + 255) / 256), 256, 0, s>>>(key, src, nq, perm, psrc);
  return cudaGetLastError();
}

}  // namespace fg
