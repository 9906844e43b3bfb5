// Depth-first search queries: a query type of the framework (Sec. 3 lists DFSs
// among the supported queries). Query q is the recursive preorder from src[q]
// with out-neighbours in the graph's arc order; disc[v] = the rank at which v
// is discovered (UINT32_MAX = not reached).
//
// A DFS is a chain of dependent steps, so the parallelism is across queries:
// one warp runs one query. At each step the warp looks at 32 arcs of the
// vertex on top of the stack at once and a ballot picks the first neighbour
// not yet discovered, which is exactly the vertex the sequential scan would
// take next. The test reads a per-query bitmap of discovered vertices (one
// bit per vertex: all queries' bitmaps stay in L2), not the ranks. The top of
// the stack stays in registers; the rest of the stack (vertex, arc to resume
// from), the bitmap and the discovery ranks live in global memory, touched
// only by that warp (its own SM's L1 sees its writes).
#include <algorithm>
#include <cstdint>

#include "fg_host.h"

namespace fg {
namespace {

constexpr int kDfsThreads = 256;  // 8 queries per block

__global__ void __launch_bounds__(kDfsThreads) dfs_kernel(DevGraph g, const int32_t *__restrict__ src, int32_t nq,
                                                          uint32_t *__restrict__ disc, uint2 *__restrict__ stack,
                                                          uint32_t *__restrict__ seen_all, int *__restrict__ bad_source) {
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = ((int64_t)gridDim.x * kDfsThreads) >> 5;
  const int64_t n = g.n;
  const int64_t words = (n + 31) / 32;
  for (int64_t q = ((int64_t)blockIdx.x * kDfsThreads + threadIdx.x) >> 5; q < nq; q += nwarps) {
    uint32_t *d = disc + q * n;
    uint2 *stk = stack + q * n;
    uint32_t *seen = seen_all + q * words;  // one bit per vertex: small enough to stay in L2
    for (int64_t v = lane; v < n; v += 32) d[v] = kInf;
    for (int64_t i = lane; i < words; i += 32) seen[i] = 0u;
    __syncwarp();
    const int32_t s = __ldg(src + q);
    if (s < 0 || s >= n) {
      if (lane == 0) atomicExch(bad_source, 1);
      continue;
    }
    uint32_t u = g.intl ? (uint32_t)__ldg(g.intl + s) : (uint32_t)s;
    uint32_t e = __ldg(g.rp + u);  // next arc of u to look at
    uint32_t time = 1;
    int64_t top = 0;               // stack depth of u (entries below it are in memory)
    if (lane == 0) {
      d[u] = 0u;
      seen[u >> 5] |= 1u << (u & 31);
    }
    __syncwarp();
    while (true) {
      const uint32_t e_end = __ldg(g.rp + u + 1);
      int64_t found = -1;
      uint32_t w = 0;
      for (uint32_t base = e; base < e_end; base += 32) {
        const uint32_t k = base + lane;
        uint32_t x = 0;
        bool fresh = false;
        if (k < e_end) {
          x = __ldg(g.adj + k);
          fresh = ((seen[x >> 5] >> (x & 31)) & 1u) == 0u;
        }
        const unsigned b = __ballot_sync(0xFFFFFFFFu, fresh);
        if (b) {
          const int j = __ffs(b) - 1;
          found = (int64_t)base + j;
          w = __shfl_sync(0xFFFFFFFFu, x, j);
          break;
        }
      }
      if (found >= 0) {
        // descend: u resumes after this arc once w is finished
        if (lane == 0) {
          stk[top] = make_uint2(u, (uint32_t)found + 1u);
          d[w] = time;
          seen[w >> 5] |= 1u << (w & 31);
        }
        __syncwarp();
        ++time;
        ++top;
        u = w;
        e = __ldg(g.rp + w);
      } else {
        // u is finished: return to its parent
        if (top == 0) break;
        --top;
        uint2 p = make_uint2(0u, 0u);
        if (lane == 0) p = stk[top];
        u = __shfl_sync(0xFFFFFFFFu, p.x, 0);
        e = __shfl_sync(0xFFFFFFFFu, p.y, 0);
      }
    }
  }
}

}  // namespace
}  // namespace fg

using namespace fg;

extern "C" fg_status fg_dfs_batch(fg_graph *g, const int32_t *src, int32_t nq, uint32_t *disc_out, void *stream_v) {
  if (!g) return fail(FG_ERR_INVALID_ARG, "graph is NULL");
  if (!src || !disc_out) return fail(FG_ERR_INVALID_ARG, "src or disc_out is NULL");
  if (nq <= 0) return fail(FG_ERR_INVALID_ARG, "nq must be > 0 (got %d)", nq);
  if ((reinterpret_cast<uintptr_t>(src) & 3u) || (reinterpret_cast<uintptr_t>(disc_out) & 3u))
    return fail(FG_ERR_INVALID_ARG, "misaligned pointer");
  int dev = -1;
  CUDA_TRY(cudaGetDevice(&dev));
  if (dev != g->device)
    return fail(FG_ERR_INVALID_ARG, "the graph lives on device %d but device %d is current", g->device, dev);
  cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_v);
  const int64_t n = g->n;
  const size_t cells = (size_t)nq * (size_t)n;

  std::lock_guard<std::mutex> lk(g->mu);
  DfsWorkspace &w = g->dfs;
  CUDA_TRY(w.stack.reserve(cells * sizeof(uint2)));
  if (g->dg.orig) CUDA_TRY(w.disc.reserve(cells * sizeof(uint32_t)));
  CUDA_TRY(w.flag.reserve(sizeof(int)));
  CUDA_TRY(w.seen.reserve((size_t)nq * (size_t)((n + 31) / 32) * sizeof(uint32_t)));
  uint32_t *disc = g->dg.orig ? w.disc.as<uint32_t>() : disc_out;
  CUDA_TRY(cudaMemsetAsync(w.flag.p, 0, sizeof(int), stream));
  const int64_t blocks = std::min<int64_t>(((int64_t)nq * 32 + kDfsThreads - 1) / kDfsThreads, 152ll * 64);
  dfs_kernel<<<(unsigned)blocks, kDfsThreads, 0, stream>>>(g->dg, src, nq, disc, w.stack.as<uint2>(),
                                                           w.seen.as<uint32_t>(), w.flag.as<int>());
  CUDA_TRY(cudaGetLastError());
  if (g->dg.orig) CUDA_TRY(launch_permute_out(disc, disc_out, g->dg.orig, n, nq, stream));
  int bad = 0;
  CUDA_TRY(cudaMemcpyAsync(&bad, w.flag.p, sizeof(int), cudaMemcpyDeviceToHost, stream));
  CUDA_TRY(cudaStreamSynchronize(stream));
  if (bad) return fail(FG_ERR_INVALID_ARG, "a source id is out of range");
  return FG_OK;
}
