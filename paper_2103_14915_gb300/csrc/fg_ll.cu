// Landmark labeling (LL) on top of a batch of SSSP / BFS queries (Sec. 1;
// Sec. 6.1 runs 1,024 SSSPs from randomly chosen landmark vertices). The
// batch's rows d(s_k, .) become per-vertex labels, and a pair (u, v) is
// answered from the two labels alone:
//     est(u, v) = min over k with d(s_k, u), d(s_k, v) finite of d(s_k, u) + d(s_k, v),
// an upper bound on d(u, v) on an undirected graph, exact when a landmark lies
// on a shortest u-v path.
//
// Both kernels move bytes and do almost no arithmetic, so HBM bandwidth bounds
// them:
//   label construction  [K][n] -> [n][K] transpose through 64 x 64 shared-memory
//                       tiles (each warp reads and writes 256 contiguous bytes
//                       per row; the padded tile keeps both phases free of bank
//                       conflicts), persistent blocks that load the next tile
//                       while writing the current one; 8 * K * n bytes;
//   query               one warp per pair reads the two K-entry labels with
//                       16-byte loads (K a multiple of 4) and reduces the
//                       minimum with shuffles; 8 * K + 16 bytes per pair.
#include <algorithm>
#include <cstdint>

#include "fg_host.h"

namespace fg {
namespace {

constexpr int kT = 64;          // transpose tile
constexpr int kTRows = 8;       // thread rows per tile (block 32 x 8)
constexpr int kQThreads = 256;  // query block: 8 warps, one pair per warp at a time

// Persistent over tiles: block b takes tiles b, b + gridDim.x, ... (vertex
// tiles fastest, so neighbouring blocks read neighbouring row segments). Each
// thread holds its 16 elements of the next tile in registers, loaded while
// the current tile is written out of shared memory.
__global__ void __launch_bounds__(32 * kTRows) ll_transpose(const uint32_t *__restrict__ dist, int32_t K, int64_t n,
                                                            uint32_t *__restrict__ labels, int64_t ntv, int64_t ntiles) {
  __shared__ uint32_t tile[kT][kT + 1];
  const int tx = threadIdx.x, ty = threadIdx.y;
  constexpr int kPer = (kT / kTRows) * (kT / 32);  // elements per thread per tile
  uint32_t buf[kPer];
  auto load = [&](int64_t t) {
    const int64_t v0 = (t % ntv) * kT;
    const int64_t k0 = (t / ntv) * kT;
#pragma unroll
    for (int r = 0; r < kT / kTRows; ++r) {
      const int64_t k = k0 + ty + r * kTRows;
#pragma unroll
      for (int c = 0; c < kT / 32; ++c) {
        const int64_t v = v0 + tx + c * 32;
        buf[r * (kT / 32) + c] = (k < K && v < n) ? __ldcs(dist + (size_t)k * (size_t)n + (size_t)v) : 0u;
      }
    }
  };
  int64_t t = blockIdx.x;
  if (t < ntiles) load(t);
  for (; t < ntiles; t += gridDim.x) {
    __syncthreads();  // the previous tile has been written out of shared memory
#pragma unroll
    for (int r = 0; r < kT / kTRows; ++r)
#pragma unroll
      for (int c = 0; c < kT / 32; ++c) tile[ty + r * kTRows][tx + c * 32] = buf[r * (kT / 32) + c];
    __syncthreads();
    const int64_t v0 = (t % ntv) * kT;
    const int64_t k0 = (t / ntv) * kT;
    if (t + gridDim.x < ntiles) load(t + gridDim.x);  // in flight during the write-out below
#pragma unroll
    for (int r = 0; r < kT / kTRows; ++r) {
      const int64_t v = v0 + ty + r * kTRows;
#pragma unroll
      for (int c = 0; c < kT / 32; ++c) {
        const int64_t k = k0 + tx + c * 32;
        if (k < K && v < n) __stcs(labels + (size_t)v * (size_t)K + (size_t)k, tile[tx + c * 32][ty + r * kTRows]);
      }
    }
  }
}

__device__ __forceinline__ void take(uint32_t a, uint32_t b, unsigned long long &best) {
  if (a != 0xFFFFFFFFu && b != 0xFFFFFFFFu) {
    const unsigned long long d = (unsigned long long)a + (unsigned long long)b;
    best = d < best ? d : best;
  }
}

template <bool VEC>
__global__ void __launch_bounds__(kQThreads) ll_query_kernel(const uint32_t *__restrict__ labels, int64_t n, int32_t K,
                                                             const int32_t *__restrict__ pairs, int64_t Q,
                                                             unsigned long long *__restrict__ out) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (kQThreads / 32);
  for (int64_t i = ((int64_t)blockIdx.x * kQThreads + threadIdx.x) >> 5; i < Q; i += warps) {
    const int32_t u = __ldg(pairs + 2 * i), v = __ldg(pairs + 2 * i + 1);
    unsigned long long best = ~0ull;
    if (u >= 0 && (int64_t)u < n && v >= 0 && (int64_t)v < n) {
      const uint32_t *lu = labels + (size_t)u * (size_t)K, *lv = labels + (size_t)v * (size_t)K;
      if (VEC) {
        const uint4 *au = reinterpret_cast<const uint4 *>(lu), *av = reinterpret_cast<const uint4 *>(lv);
        for (int32_t j = lane; j < K / 4; j += 32) {
          const uint4 a = __ldg(au + j), b = __ldg(av + j);
          take(a.x, b.x, best);
          take(a.y, b.y, best);
          take(a.z, b.z, best);
          take(a.w, b.w, best);
        }
      } else {
        for (int32_t k = lane; k < K; k += 32) take(__ldg(lu + k), __ldg(lv + k), best);
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long y = __shfl_xor_sync(0xFFFFFFFFu, best, o);
      best = y < best ? y : best;
    }
    if (lane == 0) out[i] = best;
  }
}

bool aligned(const void *p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

}  // namespace
}  // namespace fg

using namespace fg;

extern "C" fg_status fg_ll_build_labels(const uint32_t *dist, int32_t K, int64_t n, uint32_t *labels,
                                        void *stream_v) {
  if (!dist || !labels) return fail(FG_ERR_INVALID_ARG, "dist or labels is NULL");
  if (K < 1 || n < 1) return fail(FG_ERR_INVALID_ARG, "K and n must be >= 1 (got %d, %lld)", K, (long long)n);
  if (!aligned(dist, 4) || !aligned(labels, 4)) return fail(FG_ERR_INVALID_ARG, "misaligned pointer");
  cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_v);
  int dev = 0, sms = 0;
  CUDA_TRY(cudaGetDevice(&dev));
  CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int64_t ntv = (n + kT - 1) / kT, ntk = ((int64_t)K + kT - 1) / kT, ntiles = ntv * ntk;
  int per_sm = 0;
  CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ll_transpose, 32 * kTRows, 0));
  const int64_t blocks = std::min<int64_t>(ntiles, (int64_t)sms * std::max(per_sm, 1));  // all resident
  ll_transpose<<<(unsigned)blocks, dim3(32, kTRows), 0, stream>>>(dist, K, n, labels, ntv, ntiles);
  CUDA_TRY(cudaGetLastError());
  return FG_OK;
}

extern "C" fg_status fg_ll_query(const uint32_t *labels, int64_t n, int32_t K, const int32_t *pairs, int64_t Q,
                                 uint64_t *est_out, void *stream_v) {
  if (!labels || (Q > 0 && (!pairs || !est_out))) return fail(FG_ERR_INVALID_ARG, "NULL argument");
  if (K < 1 || n < 1 || Q < 0)
    return fail(FG_ERR_INVALID_ARG, "K, n must be >= 1 and Q >= 0 (got %d, %lld, %lld)", K, (long long)n,
                (long long)Q);
  if (!aligned(labels, 4) || !aligned(pairs, 4) || !aligned(est_out, 8))
    return fail(FG_ERR_INVALID_ARG, "misaligned pointer");
  if (Q == 0) return FG_OK;
  cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_v);
  const int64_t blocks = std::min<int64_t>((Q + kQThreads / 32 - 1) / (kQThreads / 32), 152ll * 64);
  unsigned long long *out = reinterpret_cast<unsigned long long *>(est_out);
  if (K % 4 == 0 && aligned(labels, 16))
    ll_query_kernel<true><<<(unsigned)blocks, kQThreads, 0, stream>>>(labels, n, K, pairs, Q, out);
  else
    ll_query_kernel<false><<<(unsigned)blocks, kQThreads, 0, stream>>>(labels, n, K, pairs, Q, out);
  CUDA_TRY(cudaGetLastError());
  return FG_OK;
}
