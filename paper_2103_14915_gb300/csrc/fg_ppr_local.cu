// Personalized PageRank with sparse per-query state, for local queries (eps
// large enough that a query touches a small part of the graph). The dense
// batch (fg_ppr_batch) keeps three rows of n floats per query; here a query
// keeps only the vertices it has touched, in an open-addressing hash table of
// `cap` slots, so that far more queries fit in HBM (20 * cap bytes each
// instead of 12 * n).
//
// The push rule is the one of fg_ppr_batch (non-lazy forward push): a vertex
// v with residual r(v) >= eps * max(d(v), 1) moves alpha * r(v) into its
// estimate (FP32, compensated) and spreads (1 - alpha) * r(v) / d(v) to each
// out-neighbour (a dangling vertex returns (1 - alpha) * r(v) to the source).
// Rounds are synchronous: every vertex active at the start of a round pushes,
// and a vertex whose residual crosses its threshold during the round is
// appended to the next round's list (exactly once: after its residual was
// taken it only grows until the next round).
//
// One block per query. The table (keys, estimate, compensation, residual)
// and the two active lists live in scratch; all reads of them go through L2
// (__ldcg) because atomics from other warps update them. A warp pushes one
// active vertex at a time, its lanes walking the arcs.
#include <algorithm>
#include <cstdint>

#include "fg_host.h"

namespace fg {
namespace {

constexpr int kLocThreads = 256;
constexpr int kLocWarps = kLocThreads / 32;

struct LocalArgs {
  DevGraph g;
  const int32_t *src = nullptr;
  int32_t nq = 0;
  float alpha = 0.f, eps = 0.f;
  uint32_t cap = 0, cap_log2 = 0;   // slots per query (a power of two)
  int32_t *keys = nullptr;          // [nq][cap] internal vertex id, -1 = empty
  float *pv = nullptr, *cv = nullptr, *rv = nullptr;  // [nq][cap] estimate, compensation, residual
  uint32_t *fa = nullptr, *fb = nullptr;              // [nq][cap] active slots (this round, next round)
  int32_t *vert_out = nullptr;      // [nq][cap] original ids of the support (p > 0)
  float *p_out = nullptr;           // [nq][cap]
  int32_t *count_out = nullptr;     // [nq]; -1 = the table filled up
  double *mass_out = nullptr;       // [nq] or null
  uint32_t max_rounds = 0;
  int *bad_source = nullptr;
};

// Slot of internal vertex w in the query's table, inserting it if absent; -1
// once the table holds 3/4 of its slots (the query is then reported full).
__device__ __forceinline__ int64_t find_or_insert(int32_t *keys, uint32_t cap, uint32_t log2, uint32_t w,
                                                  uint32_t *used, int *full) {
  uint32_t h = (w * 0x9E3779B1u) >> (32 - log2);
  for (uint32_t probe = 0; probe < cap; ++probe, h = (h + 1) & (cap - 1)) {
    const int32_t k = __ldcg(keys + h);
    if (k == (int32_t)w) return h;
    if (k == -1) {
      const int32_t prev = atomicCAS(keys + h, -1, (int32_t)w);
      if (prev == -1) {
        if (atomicAdd(used, 1u) + 1u > cap - cap / 4) *full = 1;
        return h;
      }
      if (prev == (int32_t)w) return h;
    }
  }
  *full = 1;
  return -1;
}

__global__ void __launch_bounds__(kLocThreads) ppr_local_kernel(LocalArgs a) {
  __shared__ uint32_t s_na, s_nb, s_used, s_cnt;
  __shared__ int s_full;
  __shared__ int64_t s_src_slot;
  __shared__ double s_red[kLocWarps];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t q = blockIdx.x;
  const uint32_t cap = a.cap;
  int32_t *keys = a.keys + q * cap;
  float *pv = a.pv + q * cap, *cv = a.cv + q * cap, *rv = a.rv + q * cap;
  uint32_t *fa = a.fa + q * cap, *fb = a.fb + q * cap;
  const float alpha = a.alpha, beta = 1.0f - a.alpha, eps = a.eps;

  for (uint32_t i = tid; i < cap; i += kLocThreads) {
    keys[i] = -1;
    pv[i] = 0.f;
    cv[i] = 0.f;
    rv[i] = 0.f;
  }
  if (tid == 0) {
    s_na = 0;
    s_used = 0;
    s_full = 0;
    s_src_slot = -1;
  }
  __syncthreads();
  const int32_t s = __ldg(a.src + q);
  const bool ok = s >= 0 && (int64_t)s < (int64_t)a.g.n;
  if (!ok) {
    if (tid == 0) {
      atomicExch(a.bad_source, 1);
      a.count_out[q] = 0;
      if (a.mass_out) a.mass_out[q] = 0.0;
    }
    return;
  }
  const uint32_t s_int = a.g.intl ? (uint32_t)__ldg(a.g.intl + s) : (uint32_t)s;
  if (tid == 0) {
    const int64_t slot = find_or_insert(keys, cap, a.cap_log2, s_int, &s_used, &s_full);
    s_src_slot = slot;
    if (slot >= 0) {
      __stcg(rv + slot, 1.0f);
      const uint32_t ds = __ldg(a.g.rp + s_int + 1) - __ldg(a.g.rp + s_int);
      if (1.0f >= eps * (float)(ds ? ds : 1u)) {
        fa[0] = (uint32_t)slot;
        s_na = 1;
      }
    }
  }
  __syncthreads();
  const int64_t src_slot = s_src_slot;

  for (uint32_t round = 0; round < a.max_rounds; ++round) {
    const uint32_t na = s_na;
    if (na == 0 || s_full) break;
    if (tid == 0) s_nb = 0;
    __syncthreads();
    for (uint32_t i = warp; i < na; i += kLocWarps) {
      const uint32_t slot = __ldcg(fa + i);
      const uint32_t v = (uint32_t)__ldcg(keys + slot);
      const uint32_t a0 = __ldg(a.g.rp + v), deg = __ldg(a.g.rp + v + 1) - a0;
      float inc = 0.f;
      if (lane == 0) {
        const float rho = atomicExch(rv + slot, 0.f);
        const float p0 = __ldcg(pv + slot), c0 = __ldcg(cv + slot);
        const float y = __fsub_rn(__fmul_rn(alpha, rho), c0);
        const float t = __fadd_rn(p0, y);
        __stcg(cv + slot, __fsub_rn(__fsub_rn(t, p0), y));
        __stcg(pv + slot, t);
        inc = deg ? __fdiv_rn(__fmul_rn(beta, rho), (float)deg) : __fmul_rn(beta, rho);
      }
      inc = __shfl_sync(0xFFFFFFFFu, inc, 0);
      const uint32_t arcs = deg ? deg : 1u;  // a dangling vertex sends its share back to the source
      for (uint32_t j = lane; j < arcs; j += 32) {
        int64_t ws;
        uint32_t w;
        if (deg) {
          w = __ldg(a.g.adj + a0 + j);
          ws = find_or_insert(keys, cap, a.cap_log2, w, &s_used, &s_full);
        } else {
          w = s_int;
          ws = src_slot;
        }
        if (ws < 0) continue;  // the table is full: the query is reported as such
        const uint32_t dw = __ldg(a.g.rp + w + 1) - __ldg(a.g.rp + w);
        const float thr = eps * (float)(dw ? dw : 1u);
        const float old = atomicAdd(rv + ws, inc);
        if (old < thr && __fadd_rn(old, inc) >= thr) {
          const uint32_t pos = atomicAdd(&s_nb, 1u);
          if (pos < cap) fb[pos] = (uint32_t)ws;
        }
      }
    }
    __syncthreads();
    if (tid == 0) s_na = min(s_nb, cap);
    uint32_t *t = fa;
    fa = fb;
    fb = t;
    __syncthreads();
  }

  // the support (p > 0) with the compensation folded in, and the mass
  if (tid == 0) s_cnt = 0;
  __syncthreads();
  const bool full = s_full != 0;
  double acc = 0.0;
  for (uint32_t i = tid; i < cap; i += kLocThreads) {
    const int32_t k = __ldcg(keys + i);
    if (k < 0) continue;
    const float pf = __fsub_rn(__ldcg(pv + i), __ldcg(cv + i));
    const float rf = __ldcg(rv + i);
    acc += (double)pf + (double)rf;
    if (!full && pf > 0.f) {
      const uint32_t pos = atomicAdd(&s_cnt, 1u);
      a.vert_out[q * cap + pos] = a.g.orig ? __ldg(a.g.orig + k) : k;
      a.p_out[q * cap + pos] = pf;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xFFFFFFFFu, acc, o);
  if (lane == 0) s_red[warp] = acc;
  __syncthreads();
  if (tid == 0) {
    double m = 0.0;
    for (int w = 0; w < kLocWarps; ++w) m += s_red[w];
    if (a.mass_out) a.mass_out[q] = m;
    a.count_out[q] = full ? -1 : (int32_t)s_cnt;
  }
}

}  // namespace
}  // namespace fg

using namespace fg;

extern "C" fg_status fg_ppr_local_batch(const fg_graph *g, const int32_t *src, int32_t nq, float alpha, float eps,
                                        int32_t cap, int32_t *vert_out, float *p_out, int32_t *count_out,
                                        double *mass_out, void *stream_v) {
  if (!g) return fail(FG_ERR_INVALID_ARG, "graph is NULL");
  if (!src || !vert_out || !p_out || !count_out) return fail(FG_ERR_INVALID_ARG, "NULL argument");
  if (nq <= 0) return fail(FG_ERR_INVALID_ARG, "nq must be > 0 (got %d)", nq);
  if (!(alpha > 0.f && alpha < 1.f) || !(eps > 0.f)) return fail(FG_ERR_INVALID_ARG, "need 0 < alpha < 1 and eps > 0");
  if (cap < 64 || cap > (1 << 24) || (cap & (cap - 1)))
    return fail(FG_ERR_INVALID_ARG, "cap must be a power of two in [64, 2^24] (got %d)", cap);
  if ((reinterpret_cast<uintptr_t>(src) & 3u) || (reinterpret_cast<uintptr_t>(vert_out) & 3u) ||
      (reinterpret_cast<uintptr_t>(p_out) & 3u) || (reinterpret_cast<uintptr_t>(count_out) & 3u) ||
      (reinterpret_cast<uintptr_t>(mass_out) & 7u))
    return fail(FG_ERR_INVALID_ARG, "misaligned pointer");
  int dev = -1;
  CUDA_TRY(cudaGetDevice(&dev));
  if (dev != g->device)
    return fail(FG_ERR_INVALID_ARG, "the graph lives on device %d but device %d is current", g->device, dev);
  cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_v);
  const size_t cells = (size_t)nq * (size_t)cap;
  unsigned char *scratch = nullptr;
  const size_t bytes = cells * (4 + 4 + 4 + 4 + 4 + 4) + 16;
  CUDA_TRY(cudaMallocAsync(reinterpret_cast<void **>(&scratch), bytes, stream));
  LocalArgs a;
  a.g = g->dg;
  a.src = src;
  a.nq = nq;
  a.alpha = alpha;
  a.eps = eps;
  a.cap = (uint32_t)cap;
  uint32_t l2 = 0;
  while ((1u << l2) < (uint32_t)cap) ++l2;
  a.cap_log2 = l2;
  a.keys = reinterpret_cast<int32_t *>(scratch);
  a.pv = reinterpret_cast<float *>(scratch + cells * 4);
  a.cv = reinterpret_cast<float *>(scratch + cells * 8);
  a.rv = reinterpret_cast<float *>(scratch + cells * 12);
  a.fa = reinterpret_cast<uint32_t *>(scratch + cells * 16);
  a.fb = reinterpret_cast<uint32_t *>(scratch + cells * 20);
  a.bad_source = reinterpret_cast<int *>(scratch + cells * 24);
  a.vert_out = vert_out;
  a.p_out = p_out;
  a.count_out = count_out;
  a.mass_out = mass_out;
  a.max_rounds = 1000000u;
  cudaError_t e = cudaMemsetAsync(a.bad_source, 0, sizeof(int), stream);
  if (e == cudaSuccess) {
    ppr_local_kernel<<<(unsigned)nq, kLocThreads, 0, stream>>>(a);
    e = cudaGetLastError();
  }
  int bad = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&bad, a.bad_source, sizeof(int), cudaMemcpyDeviceToHost, stream);
  cudaFreeAsync(scratch, stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
  CUDA_TRY(e);
  if (bad) return fail(FG_ERR_INVALID_ARG, "a source id is out of range");
  return FG_OK;
}
