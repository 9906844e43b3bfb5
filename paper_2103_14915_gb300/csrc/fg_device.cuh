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

namespace fg {

// ---------------------------------------------------------------------------
// Shared-memory staging with the Tensor Memory Accelerator's 1-D bulk copy
// (cp.async.bulk, global -> shared, no multicast) completing on an mbarrier.
// A phase of the mbarrier completes when its one expected arrival has come
// and every byte announced with expect_tx has landed. The issuing thread
// announces the exact total of the copies of a phase in ONE arrive.expect_tx
// before it issues any of them, so the phase can never complete early.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_addr(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

// Make initialised barriers (and generic-proxy writes to shared memory) visible
// to the async proxy before a bulk copy may complete on / write to them.
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.release.cta.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}

// A plain arrival (release: the caller's earlier shared-memory writes are seen
// by threads that wait for the phase this arrival completes).
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.acquire.cta.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait for the completion of the phase with the given parity.
// Returns false after watchdog_ns (the caller raises the status).
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, uint64_t watchdog_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  for (;;) {
    if (mbar_try_wait(bar, parity)) return true;
    if (global_ns() - t0 > watchdog_ns) return false;
  }
}

// 1-D bulk copy of `bytes` (a multiple of 16) from global src to shared dst
// (both 16-byte aligned), completing `bytes` transactions on bar.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

}  // namespace fg

namespace fg {

// 16-byte asynchronous copy global -> shared through L2 only (cp.async.cg);
// both addresses 16-byte aligned. Completion is per thread: a thread waits for
// its own groups with cp_async_wait<N>(), then a warp or block barrier makes
// every thread's copies visible to the others.
__device__ __forceinline__ void cp_async16_cg(void *smem_dst, const void *gmem_src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_addr(smem_dst)), "l"(gmem_src) : "memory");
}

// System-scope accesses to mapped host memory (a mailbox the host polls).
__device__ __forceinline__ uint32_t ld_volatile_sys(const uint32_t *p) {
  uint32_t v;
  asm volatile("ld.relaxed.sys.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_volatile_sys(uint32_t *p, uint32_t v) {
  asm volatile("st.relaxed.sys.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void st_volatile_sys(int32_t *p, int v) {
  asm volatile("st.relaxed.sys.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void fence_acq_rel_sys() { asm volatile("fence.acq_rel.sys;" ::: "memory"); }

// Ask L2 to fetch the line holding p (no register, no completion to wait for).
__device__ __forceinline__ void prefetch_l2(const void *p) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }

template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

}  // namespace fg
