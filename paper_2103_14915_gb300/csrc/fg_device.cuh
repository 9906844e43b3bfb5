// Device helpers: bounded grid barrier, warp scans and warp-aggregated atomics.
#pragma once

#include <cstdint>

#include "fg_internal.h"

namespace fg {

constexpr unsigned kFull = 0xFFFFFFFFu;

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned *p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ int ld_volatile_i32(const int *p) {
  return *reinterpret_cast<const volatile int *>(p);
}

// Raise a device status (first one wins) and ask every block to leave.
__device__ __forceinline__ void raise_status(Ctrl *c, int status, unsigned site = kSiteNone) {
  if (atomicCAS(&c->status, 0, status) == 0) atomicExch(&c->site, site);
  atomicExch(&c->abort, 1);
}

// Block barrier that first reconverges the calling warp: __syncthreads() is an
// aligned barrier and must be reached by whole, converged warps (a lane still
// inside a thread-0-only region must not let its warp count as arrived).
__device__ __forceinline__ void block_sync() {
  __syncwarp();
  __syncthreads();
}

// Device-wide barrier for a cooperative (co-resident) grid. Returns false if
// the batch is aborting (another block raised a status, or this block waited
// longer than watchdog_ns and raised FG_ERR_TIMEOUT). Every spin is bounded.
__device__ __forceinline__ bool grid_barrier(Ctrl *c, unsigned &gen, uint64_t watchdog_ns) {
  __shared__ int s_ok;
  block_sync();
  if (threadIdx.x == 0) {
    int ok = 1;
    const unsigned my_gen = gen;
    __threadfence();
    const unsigned arrived = atomicAdd(&c->bar_count, 1u);
    if (arrived == gridDim.x - 1) {
      atomicExch(&c->bar_count, 0u);
      __threadfence();
      atomicExch(&c->bar_gen, my_gen + 1u);
    } else {
      const uint64_t t0 = global_ns();
      unsigned spins = 0;
      while (ld_acquire_u32(&c->bar_gen) == my_gen) {
        if (ld_volatile_i32(&c->abort)) { ok = 0; break; }
        if ((++spins & 63u) == 0 && global_ns() - t0 > watchdog_ns) {
          raise_status(c, FG_ERR_TIMEOUT, kSiteBarrier);
          ok = 0;
          break;
        }
        __nanosleep(100);
      }
    }
    __threadfence();
    if (ld_volatile_i32(&c->abort)) ok = 0;
    s_ok = ok;
  }
  block_sync();
  gen += 1u;
  return s_ok != 0;
}

__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }

template <typename T>
__device__ __forceinline__ T warp_incl_scan(T x) {
  const int lane = lane_id();
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T y = __shfl_up_sync(kFull, x, o);
    if (lane >= o) x += y;
  }
  return x;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T x) {
#pragma unroll
  for (int o = 16; o; o >>= 1) x += __shfl_xor_sync(kFull, x, o);
  return x;
}

__device__ __forceinline__ uint32_t warp_min_u32(uint32_t x) { return __reduce_min_sync(kFull, x); }

// Largest lane L with excl[L] <= t (excl is the warp's non-decreasing
// exclusive prefix, excl[0] = 0 <= t).
__device__ __forceinline__ int owner_lane(uint32_t excl, uint32_t t) {
  int L = 0;
#pragma unroll
  for (int s = 16; s; s >>= 1) {
    uint32_t e = __shfl_sync(kFull, excl, L + s);
    if (e <= t) L += s;
  }
  return L;
}

__device__ __forceinline__ uint64_t umin64(uint64_t a, uint64_t b) { return a < b ? a : b; }

__device__ __forceinline__ uint32_t sat_add_u32(uint32_t a, uint32_t b) {
  uint32_t s = a + b;
  return s < a ? kInf : s;
}

}  // namespace fg
