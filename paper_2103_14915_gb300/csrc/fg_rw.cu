// Random-walk queries: a query type of the framework next to BFS, SSSP, PPR
// and DFS (Sec. 3 lists RWs among the supported queries). Walk q starts at
// src[q] and takes L steps; from vertex u it moves to the (r mod d(u))-th
// out-neighbour of u in the graph's arc order, where r is output number
// 2^32 * q + t + 1 of a SplitMix64 stream seeded with `seed` (Steele, Lea and
// Flood, 2014: state advanced by the golden gamma, then a mix with shifts 30,
// 27, 31). A vertex without out-arcs ends the walk.
//
// Every walk is independent, so one thread runs one walk; the graph's arcs
// are read in the internal (partition-major) order, which keeps each vertex's
// arc order. Each step is two dependent gathers (the vertex's arc range, then
// the chosen arc), so the kernel is bound by memory latency with many walks
// in flight. The walk-major output is staged 32 steps at a time in a
// shared-memory tile so that every row segment is written as one contiguous
// 128-byte piece.
#include <cstdint>

#include "fg_host.h"

namespace fg {
namespace {

constexpr int kRwThreads = 128;  // walks per block
constexpr int kChunk = 32;       // path entries staged per walk before a write-out

__device__ __forceinline__ uint64_t splitmix64_at(uint64_t seed, uint64_t k) {
  uint64_t z = seed + k * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__global__ void __launch_bounds__(kRwThreads) rw_kernel(DevGraph g, const int32_t *__restrict__ src, int32_t nq,
                                                        int32_t L, uint64_t seed, int32_t *__restrict__ paths) {
  __shared__ int32_t tile[kRwThreads][kChunk + 1];
  const int64_t q0 = (int64_t)blockIdx.x * kRwThreads;
  const int64_t q = q0 + threadIdx.x;
  int64_t u = -1;  // current vertex (internal id), -1 once the walk has ended
  if (q < nq) {
    const int32_t s = __ldg(src + q);
    if (s >= 0 && s < g.n) u = g.intl ? (int64_t)__ldg(g.intl + s) : (int64_t)s;
  }
  const int64_t row_len = (int64_t)L + 1;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int64_t t0 = 0; t0 < row_len; t0 += kChunk) {
    // path entries t0 .. t0 + 31 of this walk; entry t + 1 is the vertex after step t
    for (int j = 0; j < kChunk; ++j) {
      const int64_t t = t0 + j;
      if (t >= row_len) break;
      if (t > 0 && u >= 0) {
        const uint32_t e0 = __ldg(g.rp + u), e1 = __ldg(g.rp + u + 1);
        const uint32_t d = e1 - e0;
        if (d == 0) {
          u = -1;
        } else {
          const uint64_t r = splitmix64_at(seed, ((uint64_t)(uint32_t)q << 32) + (uint64_t)(t - 1) + 1ull);
          u = __ldg(g.adj + e0 + (uint32_t)(r % d));
        }
      }
      tile[threadIdx.x][j] = u < 0 ? -1 : (g.orig ? __ldg(g.orig + u) : (int32_t)u);
    }
    __syncthreads();
    // write-out: warp w takes rows w, w + 4, ...; lane j writes entry t0 + j
    const int64_t cols = row_len - t0 < kChunk ? row_len - t0 : kChunk;
    for (int r = warp; r < kRwThreads; r += kRwThreads / 32) {
      const int64_t qr = q0 + r;
      if (qr < nq && lane < cols) paths[qr * row_len + t0 + lane] = tile[r][lane];
    }
    __syncthreads();
  }
}

}  // namespace
}  // namespace fg

using namespace fg;

extern "C" fg_status fg_rw_batch(const fg_graph *g, const int32_t *src, int32_t nq, int32_t length, uint64_t seed,
                                 int32_t *paths_out, void *stream_v) {
  if (!g) return fail(FG_ERR_INVALID_ARG, "graph is NULL");
  if (!src || !paths_out) return fail(FG_ERR_INVALID_ARG, "src or paths_out is NULL");
  if (nq <= 0 || length < 0) return fail(FG_ERR_INVALID_ARG, "nq must be > 0 and length >= 0 (got %d, %d)", nq, length);
  if ((reinterpret_cast<uintptr_t>(src) & 3u) || (reinterpret_cast<uintptr_t>(paths_out) & 3u))
    return fail(FG_ERR_INVALID_ARG, "misaligned pointer");
  int dev = -1;
  CUDA_TRY(cudaGetDevice(&dev));
  if (dev != g->device)
    return fail(FG_ERR_INVALID_ARG, "the graph lives on device %d but device %d is current", g->device, dev);
  cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_v);
  const unsigned blocks = (unsigned)((nq + kRwThreads - 1) / kRwThreads);
  rw_kernel<<<blocks, kRwThreads, 0, stream>>>(g->dg, src, nq, length, seed, paths_out);
  CUDA_TRY(cudaGetLastError());
  return FG_OK;
}
