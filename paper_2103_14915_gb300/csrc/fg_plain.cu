// Plain per-query form (the baseline the buffered engine is compared with):
// one query at a time, ordinary whole-graph frontier iterations -- Bellman-Ford
// style relaxation for SSSP (= level-synchronous top-down BFS with unit
// weights) and Jacobi-style forward push for PPR. One cooperative launch per
// query; a device-wide barrier separates iterations.
#include "fg_device.cuh"

namespace fg {

constexpr int kPlainThreads = 256;

__device__ __forceinline__ void append_frontier(bool add, uint32_t v, uint32_t *next, uint32_t *nsize) {
  const unsigned m = __ballot_sync(kFull, add);
  if (m == 0) return;
  const int lane = lane_id(), leader = __ffs(m) - 1;
  uint32_t base = 0;
  if (lane == leader) base = atomicAdd(nsize, (unsigned)__popc(m));
  base = __shfl_sync(kFull, base, leader);
  if (add) next[base + __popc(m & ((1u << lane) - 1u))] = v;
}

template <int QT>
__global__ void __launch_bounds__(kPlainThreads) plain_kernel(PlainArgs a) {
  const DevGraph &g = a.g;
  Ctrl *c = a.ctrl;
  unsigned gen = *reinterpret_cast<volatile unsigned *>(&c->bar_gen);
  const uint32_t n = (uint32_t)g.n;
  const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x, nthr = gridDim.x * blockDim.x;
  const int lane = lane_id();
  const uint32_t gwarp = tid >> 5, nwarps = nthr >> 5;
  constexpr bool kPPR = (QT == Q_PPR);
  const int32_t s_orig = a.src[a.q];
  const bool src_ok = s_orig >= 0 && s_orig < g.n;
  const uint32_t s = src_ok ? (g.intl ? (uint32_t)g.intl[s_orig] : (uint32_t)s_orig) : 0u;
  const float alpha = a.alpha, beta = 1.0f - a.alpha, eps = a.eps;
  unsigned long long edges = 0;

  for (uint32_t i = tid; i < n; i += nthr) {
    if (kPPR) {
      a.rr[i] = 0.f; a.pp[i] = 0.f; a.cc[i] = 0.f;
    } else {
      a.dist[i] = kInf;
    }
    a.stamp[i] = 0u;
  }
  if (!grid_barrier(c, gen, a.watchdog_ns)) return;
  if (tid == 0) {
    if (!src_ok) raise_status(c, FG_ERR_INVALID_ARG, kSiteSource);
    a.sizes[0] = 0u; a.sizes[1] = 0u; a.sizes[2] = 0u;
    if (kPPR) {
      a.rr[s] = 1.0f;
      const uint32_t d = g.rp[s + 1] - g.rp[s];
      if (1.0f >= eps * (float)(d ? d : 1u)) { a.front[0][0] = s; a.sizes[0] = 1u; }
    } else {
      a.dist[s] = 0u;
      a.front[0][0] = s;
      a.sizes[0] = 1u;
    }
  }
  if (!grid_barrier(c, gen, a.watchdog_ns)) return;

  for (uint32_t it = 0;; ++it) {
    const uint32_t *F = a.front[it & 1u];
    uint32_t *N = a.front[(it + 1u) & 1u];
    const uint32_t nF = *reinterpret_cast<volatile uint32_t *>(&a.sizes[it % 3u]);
    uint32_t *nsize = &a.sizes[(it + 1u) % 3u];
    if (nF == 0u) break;
    if (it >= a.max_rounds) {
      if (tid == 0) raise_status(c, FG_ERR_TIMEOUT, kSiteRounds);
      break;
    }
    if (tid == 0) a.sizes[(it + 2u) % 3u] = 0u;
    const uint32_t stamp = it + 1u;
    for (uint32_t c0 = gwarp * 32u; c0 < nF; c0 += nwarps * 32u) {
      const uint32_t idx = c0 + (uint32_t)lane;
      const bool valid = idx < nF;
      uint32_t v = 0, a0 = 0, deg = 0, dv = 0;
      float inc_l = 0.f;
      if (valid) {
        v = __ldcg(F + idx);
        a0 = g.rp[v];
        deg = g.rp[v + 1] - a0;
        if (kPPR) {
          const float rho = atomicExch(&a.rr[v], 0.f);
          const float pv = __ldcg(a.pp + v), cv = __ldcg(a.cc + v);
          const float y = __fsub_rn(__fmul_rn(alpha, rho), cv);
          const float t = __fadd_rn(pv, y);
          __stcg(a.cc + v, __fsub_rn(__fsub_rn(t, pv), y));
          __stcg(a.pp + v, t);
          inc_l = deg ? __fdiv_rn(__fmul_rn(beta, rho), (float)deg) : __fmul_rn(beta, rho);
        } else {
          dv = __ldcg(&a.dist[v]);
        }
      }
      const uint32_t arcs = valid ? (kPPR ? (deg ? deg : 1u) : deg) : 0u;
      const uint32_t incl = warp_incl_scan(arcs);
      const uint32_t exd = incl - arcs;
      const uint32_t tot = __shfl_sync(kFull, incl, 31);
      edges += tot;
      for (uint32_t j = 0; j < tot; j += 32) {
        const uint32_t t = j + (uint32_t)lane;
        const bool has = t < tot;
        const int L = owner_lane(exd, has ? t : 0u);
        const uint32_t eL = __shfl_sync(kFull, a0, L) + (t - __shfl_sync(kFull, exd, L));
        const uint32_t degL = __shfl_sync(kFull, deg, L);
        const uint32_t du = __shfl_sync(kFull, dv, L);
        const float inc = __shfl_sync(kFull, inc_l, L);
        bool add = false;
        uint32_t u = 0;
        if (has) {
          if (kPPR) {
            u = degL ? g.adj[eL] : s;
            const uint32_t dd = g.rp[u + 1] - g.rp[u];
            const float thr = eps * (float)(dd ? dd : 1u);
            const float old = atomicAdd(&a.rr[u], inc);
            add = old < thr && __fadd_rn(old, inc) >= thr;
          } else {
            u = g.adj[eL];
            const uint32_t wgt = (QT == Q_BFS || g.wt == nullptr) ? 1u : g.wt[eL];
            const uint64_t s64 = (uint64_t)du + wgt;
            uint32_t nd;
            if (s64 >= (uint64_t)kInf) {
              atomicCAS(&c->status, 0, (int)FG_ERR_OVERFLOW);
              nd = kInf - 1u;
            } else {
              nd = (uint32_t)s64;
            }
            const uint32_t old = atomicMin(&a.dist[u], nd);
            add = nd < old && atomicExch(&a.stamp[u], stamp) != stamp;
          }
        }
        append_frontier(add, u, N, nsize);
      }
    }
    if (!grid_barrier(c, gen, a.watchdog_ns)) return;
    if (tid == 0) atomicAdd(&c->rounds, 1ull);
  }
  // copy the query's row out in original vertex order
  for (uint32_t i = tid; i < n; i += nthr) {
    const uint32_t gi = g.orig ? (uint32_t)g.orig[i] : i;
    if (kPPR) {
      a.out_p[gi] = __ldcg(a.pp + i);
      a.out_r[gi] = __ldcg(a.rr + i);
      a.out_c[gi] = __ldcg(a.cc + i);
    } else {
      a.out_u32[gi] = __ldcg(a.dist + i);
    }
  }
  // edges is warp-uniform (every lane added each chunk's total)
  if (lane == 0 && edges) atomicAdd(&c->edges, edges);
}

static const void *plain_fn(int qtype) {
  switch (qtype) {
    case Q_SSSP: return (const void *)plain_kernel<Q_SSSP>;
    case Q_BFS: return (const void *)plain_kernel<Q_BFS>;
    default: return (const void *)plain_kernel<Q_PPR>;
  }
}

cudaError_t plain_grid_size(int *blocks, int *threads) {
  int per_sm = 0, dev = 0, sms = 0;
  cudaError_t e;
  int best = 1 << 30;
  for (int qt = 0; qt < 3; ++qt) {
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, plain_fn(qt), kPlainThreads, 0)) != cudaSuccess)
      return e;
    best = per_sm < best ? per_sm : best;
  }
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  if (best < 1) return cudaErrorInvalidConfiguration;
  *threads = kPlainThreads;
  *blocks = best * sms;
  return cudaSuccess;
}

cudaError_t launch_plain(const PlainArgs &a, int blocks, int threads, cudaStream_t s) {
  PlainArgs copy = a;
  void *args[] = {(void *)&copy};
  return cudaLaunchCooperativeKernel(plain_fn(a.qtype), dim3(blocks), dim3(threads), args, 0, s);
}

}  // namespace fg
