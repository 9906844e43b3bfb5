// Sweep cuts over PPR vectors: the conductance step of the network community
// profile (NCP) application, which runs PPRs from a random sample of seed
// vertices (Sec. 1; Sec. 6.1 seeds 0.01% of the vertices). For query q the
// vertices with p(v) > 0 are ordered by the FP32 key p(v) / max(d(v), 1),
// largest first, ties by smaller original id; for each prefix S_k of the first
// `top` of them the kernel writes the conductance
//     phi(S_k) = cut(S_k) / min(vol(S_k), vol(V) - vol(S_k)),
// vol = sum of out-degrees, cut = arcs from S_k to the rest; and, across all
// queries of the call, the profile NCP(k) = min over queries of phi(S_k).
//
// One block per query (with few queries, several blocks per query, below):
//   1. select  one pass over the row: vertex v gets the 64-bit sort key
//              (~key bits << 32 | v), unique, ascending = key descending then
//              id ascending; keys that may still be among the `top` smallest
//              go into a shared-memory buffer, which is cut back to exactly
//              `top` keys (radix select over 8-bit digits inside the buffer)
//              whenever the next tile might not fit, after which only keys
//              below the `top`-th are admitted. With the tiles in a scrambled
//              order about top * (1 + ln(#positive / top)) keys are admitted;
//              a vertex whose key must round below the threshold is skipped
//              before the division (an FP32 test with a stated bound);
//   2. sort    bitonic sort of the kept keys;
//   3. rank    a shared-memory hash from each chosen vertex's internal id to
//              its sweep rank; the neighbours ranked before a vertex are
//              counted by one lane (light vertex), one warp (medium) or the
//              whole block (a hub of more than 4,096 arcs);
//   4. scan    prefix sums of d(v) - 2 * inside(v) and of d(v) give cut and vol
//              exactly in int64; phi = cut / den in FP64.
// When there are too few rows to give every SM two blocks, each row is split
// into segments: a block per segment runs step 1 and leaves its top keys in
// scratch (from the stream-ordered allocator), and a block per row merges the
// segments' keys through the same buffer and runs steps 2-4. The kept set
// does not depend on the split.
//
// The row read (p from HBM, 4 B per vertex, float4 loads one tile ahead; the
// degree table, shared by all queries, mostly from L2) is the traffic; steps
// 2-4 touch only shared memory and the chosen vertices' adjacency.
#include <algorithm>
#include <cstdint>
#include <cstdio>
#include <mutex>

#include "fg_host.h"

namespace fg {
namespace {

constexpr int kThreads = 512;                   // 16 warps
constexpr int kWarps = kThreads / 32;
constexpr int kMaxTop = FG_NCP_MAX_TOP;         // 4096
constexpr int kCap = 2 * kMaxTop;               // candidate buffer (64-bit entries)
constexpr int kHash = 2 * kMaxTop;              // hash slots (load <= 1/2)
constexpr int kHashLog2 = 13;
constexpr uint32_t kEmpty = 0xFFFFFFFFu;
static_assert(kHash == (1 << kHashLog2), "hash size");
static_assert(kCap * 8 == kHash * 8, "the hash reuses the candidate buffer");

// dynamic shared memory
//   A: cand[kCap] u64 (steps 1-2), then hash keys[kHash] u32 + vals[kHash] u32 (step 3)
//   B + C: the cut-back copy tmp[kMaxTop] u64 (step 1); then
//   B: ord[kMaxTop] u32: internal id, then d - 2*inside (steps 3-4)
//   C: dgs[kMaxTop] u32 (degrees of the chosen vertices)
constexpr size_t kBytesA = (size_t)kCap * 8;
constexpr size_t kBytesB = (size_t)kMaxTop * 4;
constexpr size_t kBytesC = (size_t)kMaxTop * 4;
constexpr size_t kSmem = kBytesA + kBytesB + kBytesC;
static_assert(kBytesB + kBytesC >= (size_t)kMaxTop * 8, "regions B + C hold the cut-back copy");

struct NcpArgs {
  const float *p = nullptr;        // [nq][n] original order
  const uint32_t *deg = nullptr;   // [n] out-degree, original order
  const uint32_t *rp = nullptr;    // [n+1] internal order
  const uint32_t *adj = nullptr;   // [m] internal ids
  const int32_t *intl = nullptr;   // original -> internal, or null (identity)
  int64_t n = 0;
  uint64_t m = 0;
  int32_t top = 0;
  int32_t *order = nullptr;        // [nq][top] or null
  double *phi = nullptr;           // [nq][top] or null
  int32_t *count = nullptr;        // [nq] or null
  unsigned long long *ncp = nullptr;  // [top] encoded profile, or null
};

// Sort key of a vertex: FP32 bit pattern of p / max(d, 1) plus one (bit
// patterns of non-negative floats order as the floats do); 0 = not a
// candidate (p not > 0, which also rejects NaN).
__device__ __forceinline__ uint32_t key_enc(float p, uint32_t d) {
  if (!(p > 0.f)) return 0u;
  const float k = __fdiv_rn(p, __uint2float_rn(d > 0u ? d : 1u));
  return __float_as_uint(k) + 1u;
}

// Order-preserving map of a double onto uint64 (for atomicMin), and back.
__device__ __forceinline__ unsigned long long dbl_enc(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}
__device__ __forceinline__ double dbl_dec(unsigned long long e) {
  const unsigned long long b = (e >> 63) ? (e & 0x7FFFFFFFFFFFFFFFull) : ~e;
  return __longlong_as_double((long long)b);
}

// Inclusive prefix sum within a warp.
template <typename T>
__device__ __forceinline__ T warp_prefix_incl(T x, int lane) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const T y = __shfl_up_sync(0xFFFFFFFFu, x, o);
    if (lane >= o) x += y;
  }
  return x;
}

constexpr int kVecPerTile = 1;                    // float4 row loads per thread per tile
constexpr int kSlots = 4 * kVecPerTile;            // row elements per thread per tile
constexpr int kTile = kThreads * kSlots;           // row elements per tile
// After a cut the buffer holds `top` <= kMaxTop keys; the room left above that
// decides how often the buffer is cut (a cut is a radix select over it).
static_assert(kCap - kTile >= kMaxTop + kTile, "after a cut, at least one full tile of admissions fits before the next");

// Row elements of tile t held by this thread: slot e. Vector form (n a
// multiple of 4): float4 / uint4 loads, element
// 4 * (t * kVecPerTile * kThreads + (e / 4) * kThreads + tid) + e % 4; scalar
// form: t * kTile + e * kThreads + tid. Each warp's addresses are contiguous.
template <bool VEC>
__device__ __forceinline__ int64_t slot_index(int64_t t, int e) {
  if (VEC) return 4 * (t * kVecPerTile * kThreads + (int64_t)(e >> 2) * kThreads + threadIdx.x) + (e & 3);
  return t * kTile + (int64_t)e * kThreads + threadIdx.x;
}

template <bool VEC>
__device__ __forceinline__ void load_tile(const float *prow, const uint32_t *deg, int64_t n, int64_t t,
                                          float (&pv)[kSlots], uint32_t (&dv)[kSlots]) {
  if (VEC) {
#pragma unroll
    for (int h = 0; h < kVecPerTile; ++h) {
      const int64_t v = slot_index<true>(t, 4 * h);
      float4 p4 = make_float4(0.f, 0.f, 0.f, 0.f);
      uint4 d4 = make_uint4(0u, 0u, 0u, 0u);
      if (v < n) {  // n is a multiple of 4: the whole vector is in the row
        p4 = __ldg(reinterpret_cast<const float4 *>(prow + v));
        d4 = __ldg(reinterpret_cast<const uint4 *>(deg + v));
      }
      pv[4 * h] = p4.x; pv[4 * h + 1] = p4.y; pv[4 * h + 2] = p4.z; pv[4 * h + 3] = p4.w;
      dv[4 * h] = d4.x; dv[4 * h + 1] = d4.y; dv[4 * h + 2] = d4.z; dv[4 * h + 3] = d4.w;
    }
  } else {
#pragma unroll
    for (int e = 0; e < kSlots; ++e) {
      const int64_t v = slot_index<false>(t, e);
      pv[e] = v < n ? __ldg(prow + v) : 0.f;
      dv[e] = v < n ? __ldg(deg + v) : 0u;
    }
  }
}

// Sort key of a candidate: ascending order = key descending, id ascending.
// Unique per vertex, so "the top smallest sort keys" is exact with no ties.
__device__ __forceinline__ unsigned long long sort_key(uint32_t enc, uint32_t v) {
  return ((unsigned long long)(~enc) << 32) | v;
}

struct Stream {
  unsigned long long *buf;  // [kCap] candidates (region A)
  unsigned long long *tmp;  // [kMaxTop] (regions B + C)
  uint32_t *h;              // [256] digit histogram
  uint32_t *wsum;           // [kWarps]
  uint32_t *n_buf;          // candidates held
  uint32_t *n_tmp;
  unsigned long long *thr;  // keys >= thr cannot rank among the top any more
  uint32_t *sel;            // [2] bucket of the top-th key, keys below that bucket
};

// Cut the buffer back to its T smallest keys (block-wide; B = held > T).
// Radix select over the eight 8-bit digits of the 64-bit keys, from the top:
// each pass narrows the prefix of the T-th smallest key; after the last one
// the prefix is that key itself (keys are unique). The buffer keeps the keys
// <= it, and from then on the stream admits only keys below it.
__device__ void cut_back(const Stream &st, uint32_t T) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t B = *st.n_buf;
  unsigned long long prefix = 0;
  uint32_t below = 0;
  for (int shift = 56; shift >= 0; shift -= 8) {
    for (int i = tid; i < 256; i += kThreads) st.h[i] = 0u;
    __syncthreads();
    // the leading digits of the held keys fall into few bins: lanes with the
    // same bin add their count through one atomic (else they serialise)
    for (uint32_t base = 0; base < B; base += kThreads) {
      const uint32_t i = base + tid;
      uint32_t bin = 0xFFFFFFFFu;
      if (i < B) {
        const unsigned long long k = st.buf[i];
        if (shift == 56 || (k >> (shift + 8)) == prefix) bin = (uint32_t)((k >> shift) & 255u);
      }
      const unsigned grp = __match_any_sync(0xFFFFFFFFu, bin);
      if (bin != 0xFFFFFFFFu && lane == __ffs(grp) - 1) atomicAdd(&st.h[bin], (uint32_t)__popc(grp));
    }
    __syncthreads();
    // inclusive prefix over the 256 bins (threads 0..255, warps 0..7)
    uint32_t c = tid < 256 ? st.h[tid] : 0u;
    uint32_t incl = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
      if (lane >= o) incl += y;
    }
    if (lane == 31 && warp < 8) st.wsum[warp] = incl;
    __syncthreads();
    if (tid < 256) {
      uint32_t off = below;
      for (int w = 0; w < warp; ++w) off += st.wsum[w];
      const uint32_t hi = off + incl, lo = hi - c;
      if (lo < T && hi >= T) {
        st.sel[0] = (uint32_t)tid;
        st.sel[1] = lo;
      }
    }
    __syncthreads();
    prefix = (prefix << 8) | st.sel[0];
    below = st.sel[1];
    __syncthreads();  // sel and h are rewritten by the next digit
  }
  const unsigned long long kth = prefix;  // the T-th smallest key
  if (tid == 0) *st.n_tmp = 0u;
  __syncthreads();
  for (uint32_t i = tid; i < B; i += kThreads) {
    const unsigned long long k = st.buf[i];
    if (k <= kth) {
      const uint32_t pos = atomicAdd(st.n_tmp, 1u);
      if (pos < (uint32_t)kMaxTop) st.tmp[pos] = k;
    }
  }
  __syncthreads();
  const uint32_t kept = min(*st.n_tmp, (uint32_t)kMaxTop);
  for (uint32_t i = tid; i < kept; i += kThreads) st.buf[i] = st.tmp[i];
  if (tid == 0) {
    *st.n_buf = kept;
    *st.thr = kth;
  }
  __syncthreads();
}

// Admission of one tile (block-wide): each thread offers up to kSlots keys
// (bit e of `mask` set = key[e] is below the threshold); admitted keys are
// appended to the buffer, and the barrier that ends the tile decides,
// uniformly, whether the buffer must be cut before the next tile.
__device__ __forceinline__ void admit_tile(const Stream &st, uint32_t T, const unsigned long long (&key)[kSlots],
                                           unsigned mask) {
  const int lane = threadIdx.x & 31;
  uint32_t held_after = 0;  // lane 0: the count right after this warp's last append
  if (__any_sync(0xFFFFFFFFu, mask != 0u)) {  // most tiles admit nothing once the buffer is full
#pragma unroll
    for (int e = 0; e < kSlots; ++e) {
      const bool take = (mask >> e) & 1u;
      const unsigned bal = __ballot_sync(0xFFFFFFFFu, take);
      if (bal) {
        uint32_t pos = 0;
        if (lane == 0) {
          pos = atomicAdd(st.n_buf, (uint32_t)__popc(bal));
          held_after = max(held_after, pos + (uint32_t)__popc(bal));
        }
        pos = __shfl_sync(0xFFFFFFFFu, pos, 0) + (uint32_t)__popc(bal & ((1u << lane) - 1u));
        if (take && pos < (uint32_t)kCap) st.buf[pos] = key[e];
      }
    }
  }
  // The last append of the tile saw the final count. (Reading the count after
  // a plain barrier would race with the next tile's appends.)
  if (__syncthreads_or(held_after > (uint32_t)(kCap - kTile))) cut_back(st, T);
}

__device__ __forceinline__ void stream_begin(const Stream &st) {
  if (threadIdx.x == 0) {
    *st.n_buf = 0u;
    *st.thr = ~0ull;  // every key is admitted until the first cut (real keys are below 2^64 - 2^32)
  }
  __syncthreads();
}

// The FP32 key value of the threshold (0 while every key is admitted).
__device__ __forceinline__ float thr_key(unsigned long long thr) {
  if (thr == ~0ull) return 0.f;
  const uint32_t enc = ~(uint32_t)(thr >> 32);
  return __uint_as_float(enc - 1u);
}

// Steps 1-2 over tiles [tlo, thi) of a row: every vertex whose sort key may
// still be among the T smallest is kept (the buffer holds at most T after the
// final cut). Tiles are visited in a scrambled order: step i takes tile
// tlo + (i * odd) mod P, P = the range rounded up to a power of two (a
// bijection; steps past the range load nothing), so keys that drift along the
// vertex ids (degree correlates with id in R-MAT numbering) do not keep
// beating the threshold.
//
// Most vertices end far below the threshold key K, and the exact key needs an
// IEEE division. A vertex is skipped without it when p < (K (1 - 2^-20)) * d
// in FP32 (three roundings of at most 2^-24 each: the conversion of d and the
// two products, so p / d < K (1 - 2^-21) and the rounded key is below K); the
// test is used only while the products are normal and finite. Every other
// vertex gets its exact key.
template <bool VEC>
__device__ void stream_row(const NcpArgs &a, const float *prow, const Stream &st, uint32_t T, int64_t tlo,
                           int64_t thi) {
  const int64_t n = a.n;
  int64_t P = 1;
  while (P < thi - tlo) P <<= 1;
  auto tile_at = [P, tlo](int64_t i) {
    return tlo + (int64_t)(((uint64_t)i * 0x9E3779B97F4A7C15ull) & (uint64_t)(P - 1));
  };
  const int64_t hi_elem = thi * kTile;  // elements of tiles >= thi belong to another segment
  float pc[kSlots];
  uint32_t dc[kSlots];
  load_tile<VEC>(prow, a.deg, n, tile_at(0) < thi ? tile_at(0) : (n + kTile) / kTile + 1, pc, dc);
  for (int64_t i = 0; i < P; ++i) {
    const int64_t t = tile_at(i);
    float pn[kSlots] = {};
    uint32_t dn[kSlots] = {};
    if (i + 1 < P) {
      const int64_t tn = tile_at(i + 1);
      if (tn < thi) load_tile<VEC>(prow, a.deg, n, tn, pn, dn);  // in flight while tile t is filtered
    }
    const unsigned long long thr = *st.thr;
    // Kc = K (1 - 2^-20), rounded; used only while it is a normal number, so
    // that Kc * d (d >= 1) is normal too (the products stay finite: checked)
    const float Kc = __fmul_rn(thr_key(thr), 0x1.ffffe0p-1f);
    const bool filt = Kc >= 1.17549435e-38f;  // FLT_MIN
    unsigned long long key[kSlots];
    unsigned mask = 0;  // slots of this thread that are admitted
#pragma unroll
    for (int e = 0; e < kSlots; ++e) {
      const int64_t v = slot_index<VEC>(t, e);
      key[e] = ~0ull;
      if (t >= thi || v >= hi_elem || !(pc[e] > 0.f)) continue;
      if (filt) {
        const float lim = __fmul_rn(Kc, __uint2float_rn(dc[e] > 0u ? dc[e] : 1u));
        if (lim <= 3.40282347e+38f && pc[e] < lim) continue;
      }
      const uint32_t enc = key_enc(pc[e], dc[e]);
      key[e] = sort_key(enc, (uint32_t)v);
      if (key[e] < thr) mask |= 1u << e;
    }
    admit_tile(st, T, key, mask);
#pragma unroll
    for (int e = 0; e < kSlots; ++e) {
      pc[e] = pn[e];
      dc[e] = dn[e];
    }
  }
  if (*st.n_buf > T) cut_back(st, T);
}

// Merge: stream `count` keys (segments' survivors, ~0 = padding) through the
// same buffer; at most T are held afterwards.
__device__ void stream_keys(const unsigned long long *keys, int64_t count, const Stream &st, uint32_t T) {
  for (int64_t base = 0; base < count; base += kTile) {
    const unsigned long long thr = *st.thr;
    unsigned long long key[kSlots];
    unsigned mask = 0;
#pragma unroll
    for (int e = 0; e < kSlots; ++e) {
      const int64_t i = base + (int64_t)e * kThreads + threadIdx.x;
      key[e] = i < count ? __ldcg(keys + i) : ~0ull;
      if (key[e] < thr) mask |= 1u << e;
    }
    admit_tile(st, T, key, mask);
  }
  if (*st.n_buf > T) cut_back(st, T);
}

struct Smem {
  unsigned long long *cand;
  uint32_t *hkey, *hval, *ord, *dgs;
};

__device__ __forceinline__ Smem carve(unsigned char *smem) {
  Smem m;
  m.cand = reinterpret_cast<unsigned long long *>(smem);
  m.hkey = reinterpret_cast<uint32_t *>(smem);
  m.hval = m.hkey + kHash;
  m.ord = reinterpret_cast<uint32_t *>(smem + kBytesA);
  m.dgs = reinterpret_cast<uint32_t *>(smem + kBytesA + kBytesB);
  return m;
}

// Steps 2-4 for row q, with the L (<= top) kept keys in cand[0, L).
__device__ void finish_row(const NcpArgs &a, int64_t q, uint32_t L, const Smem &m);

// One block per row: the whole row streamed, then steps 2-4.
__global__ void __launch_bounds__(kThreads, 2) ncp_sweep_kernel(NcpArgs a, bool vec) {
  extern __shared__ __align__(16) unsigned char smem[];
  const Smem m = carve(smem);
  __shared__ uint32_t s_h[256], s_w32[kWarps], s_sel[2], s_n, s_m;
  __shared__ unsigned long long s_thr;
  const int64_t q = blockIdx.x;
  const Stream st{m.cand, reinterpret_cast<unsigned long long *>(smem + kBytesA), s_h, s_w32, &s_n, &s_m, &s_thr, s_sel};
  stream_begin(st);
  const int64_t ntiles = (a.n + kTile - 1) / kTile;
  if (vec) stream_row<true>(a, a.p + q * a.n, st, (uint32_t)a.top, 0, ntiles);
  else stream_row<false>(a, a.p + q * a.n, st, (uint32_t)a.top, 0, ntiles);
  finish_row(a, q, min(*st.n_buf, (uint32_t)a.top), m);
}

// `parts` blocks per row: block (q, c) keeps the top keys of segment c of row
// q and writes them to scratch[(q * parts + c) * top ...], padded with ~0.
__global__ void __launch_bounds__(kThreads, 2) ncp_select_kernel(NcpArgs a, bool vec, int parts,
                                                                 unsigned long long *scratch) {
  extern __shared__ __align__(16) unsigned char smem[];
  const Smem m = carve(smem);
  __shared__ uint32_t s_h[256], s_w32[kWarps], s_sel[2], s_n, s_m;
  __shared__ unsigned long long s_thr;
  const int64_t q = blockIdx.x / parts;
  const int c = (int)(blockIdx.x % parts);
  const Stream st{m.cand, reinterpret_cast<unsigned long long *>(smem + kBytesA), s_h, s_w32, &s_n, &s_m, &s_thr, s_sel};
  stream_begin(st);
  const int64_t ntiles = (a.n + kTile - 1) / kTile;
  const int64_t tlo = ntiles * c / parts, thi = ntiles * (c + 1) / parts;
  if (vec) stream_row<true>(a, a.p + q * a.n, st, (uint32_t)a.top, tlo, thi);
  else stream_row<false>(a, a.p + q * a.n, st, (uint32_t)a.top, tlo, thi);
  const uint32_t held = min(*st.n_buf, (uint32_t)a.top);
  unsigned long long *out = scratch + ((size_t)q * parts + c) * (size_t)a.top;
  for (uint32_t i = threadIdx.x; i < (uint32_t)a.top; i += kThreads) __stcg(out + i, i < held ? m.cand[i] : ~0ull);
}

// One block per row: merge the row's `parts` segments, then steps 2-4.
__global__ void __launch_bounds__(kThreads, 2) ncp_merge_kernel(NcpArgs a, int parts,
                                                                const unsigned long long *scratch) {
  extern __shared__ __align__(16) unsigned char smem[];
  const Smem m = carve(smem);
  __shared__ uint32_t s_h[256], s_w32[kWarps], s_sel[2], s_n, s_m;
  __shared__ unsigned long long s_thr;
  const int64_t q = blockIdx.x;
  const Stream st{m.cand, reinterpret_cast<unsigned long long *>(smem + kBytesA), s_h, s_w32, &s_n, &s_m, &s_thr, s_sel};
  stream_begin(st);
  stream_keys(scratch + (size_t)q * parts * (size_t)a.top, (int64_t)parts * a.top, st, (uint32_t)a.top);
  finish_row(a, q, min(*st.n_buf, (uint32_t)a.top), m);
}

__device__ void finish_row(const NcpArgs &a, int64_t q, uint32_t L, const Smem &m) {
  unsigned long long *cand = m.cand;
  uint32_t *hkey = m.hkey, *hval = m.hval, *ord = m.ord, *dgs = m.dgs;
  __shared__ unsigned long long s_w64[2][kWarps];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t T = (uint32_t)a.top;
  const uint32_t kmax = L;

  // ---- 2. sort ----------------------------------------------------------
  uint32_t L2 = 2;
  while (L2 < L) L2 <<= 1;
  for (uint32_t i = L + tid; i < L2; i += kThreads) cand[i] = ~0ull;
  __syncthreads();
  for (uint32_t k = 2; k <= L2; k <<= 1) {
    for (uint32_t j = k >> 1; j > 0; j >>= 1) {
      for (uint32_t i = tid; i < L2; i += kThreads) {
        const uint32_t ixj = i ^ j;
        if (ixj > i) {
          const unsigned long long x = cand[i], y = cand[ixj];
          const bool up = (i & k) == 0u;
          if ((x > y) == up) {
            cand[i] = y;
            cand[ixj] = x;
          }
        }
      }
      __syncthreads();
    }
  }

  // ---- 3. rank ----------------------------------------------------------
  int32_t *orow = a.order ? a.order + q * a.top : nullptr;
  for (uint32_t k = tid; k < kmax; k += kThreads) {
    const uint32_t v = (uint32_t)cand[k];
    if (orow) orow[k] = (int32_t)v;
    const uint32_t u = a.intl ? (uint32_t)__ldg(a.intl + v) : v;
    ord[k] = u;
    dgs[k] = __ldg(a.rp + u + 1) - __ldg(a.rp + u);
  }
  __syncthreads();  // the candidate buffer is free from here on
  for (int i = tid; i < kHash; i += kThreads) hkey[i] = kEmpty;
  __syncthreads();
  for (uint32_t k = tid; k < kmax; k += kThreads) {
    const uint32_t u = ord[k];
    uint32_t s = (u * 0x9E3779B1u) >> (32 - kHashLog2);
    for (int probe = 0; probe < kHash; ++probe, s = (s + 1) & (kHash - 1)) {
      if (atomicCAS(&hkey[s], kEmpty, u) == kEmpty) {
        hval[s] = k;
        break;
      }
    }
  }
  __syncthreads();
  // neighbours ranked before k. The sweep set mixes many light vertices with a
  // few hubs (tens of thousands of arcs), so the count is split three ways:
  // a light vertex (<= 32 arcs) is counted by one lane, so that 32 vertices'
  // load chains are in flight per warp; a medium one by its warp; a hub
  // (more than kBlockArcs arcs) by the whole block, after the rest. Every
  // thread keeps 4 arc loads in flight before it probes the hash.
  constexpr uint32_t kBlockArcs = 4096;
  constexpr int kMaxHubs = 64;
  __shared__ uint32_t s_hub[kMaxHubs], s_nhub, s_red[kWarps];
  auto ranked_before = [&](uint32_t w, uint32_t k) -> uint32_t {
    uint32_t sl = (w * 0x9E3779B1u) >> (32 - kHashLog2);
    for (int probe = 0; probe < kHash; ++probe, sl = (sl + 1) & (kHash - 1)) {
      const uint32_t hk = hkey[sl];
      if (hk == w) return hval[sl] < k ? 1u : 0u;
      if (hk == kEmpty) return 0u;
    }
    return 0u;
  };
  // arcs [b, e1) with stride `step`, 4 loads in flight per thread
  auto count_arcs = [&](uint32_t b, uint32_t e1, uint32_t step, uint32_t k) -> uint32_t {
    uint32_t inside = 0;
    for (uint32_t e = b; e < e1; e += 4 * step) {
      uint32_t w4[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) w4[j] = e + j * step < e1 ? __ldg(a.adj + e + j * step) : kEmpty;
#pragma unroll
      for (int j = 0; j < 4; ++j)
        if (w4[j] != kEmpty) inside += ranked_before(w4[j], k);
    }
    return inside;
  };
  if (tid == 0) s_nhub = 0;
  __syncthreads();
  for (uint32_t k0 = warp * 32; k0 < kmax; k0 += kWarps * 32) {
    const uint32_t k = k0 + lane;
    uint32_t e0 = 0, e1 = 0;
    if (k < kmax) {
      const uint32_t u = ord[k];
      e0 = __ldg(a.rp + u);
      e1 = __ldg(a.rp + u + 1);
    }
    const bool light = k < kmax && e1 - e0 <= 32u;
    if (light) ord[k] = (uint32_t)((int32_t)dgs[k] - 2 * (int32_t)count_arcs(e0, e1, 1u, k));
    unsigned heavy = __ballot_sync(0xFFFFFFFFu, k < kmax && !light);
    while (heavy) {
      const int j = __ffs(heavy) - 1;
      heavy &= heavy - 1;
      const uint32_t kh = k0 + j;
      const uint32_t h0 = __shfl_sync(0xFFFFFFFFu, e0, j), h1 = __shfl_sync(0xFFFFFFFFu, e1, j);
      if (h1 - h0 > kBlockArcs) {
        uint32_t slot = 0;
        if (lane == 0) slot = atomicAdd(&s_nhub, 1u);
        slot = __shfl_sync(0xFFFFFFFFu, slot, 0);
        if (slot < (uint32_t)kMaxHubs) {
          if (lane == 0) s_hub[slot] = kh;  // counted by the block below
          continue;
        }
      }
      uint32_t inside = count_arcs(h0 + lane, h1, 32u, kh);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) inside += __shfl_xor_sync(0xFFFFFFFFu, inside, o);
      if (lane == j) ord[kh] = (uint32_t)((int32_t)dgs[kh] - 2 * (int32_t)inside);
    }
  }
  __syncthreads();
  const uint32_t nhub = min(s_nhub, (uint32_t)kMaxHubs);
  for (uint32_t i = 0; i < nhub; ++i) {
    const uint32_t kh = s_hub[i];
    // ord[kh] still holds the hub's internal id: every thread reads it before the write below
    const uint32_t u = ord[kh];
    const uint32_t h0 = __ldg(a.rp + u), h1 = __ldg(a.rp + u + 1);
    uint32_t inside = count_arcs(h0 + tid, h1, kThreads, kh);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) inside += __shfl_xor_sync(0xFFFFFFFFu, inside, o);
    if (lane == 0) s_red[warp] = inside;
    __syncthreads();
    if (tid == 0) {
      uint32_t tot = 0;
      for (int w = 0; w < kWarps; ++w) tot += s_red[w];
      ord[kh] = (uint32_t)((int32_t)dgs[kh] - 2 * (int32_t)tot);
    }
    __syncthreads();
  }

  // ---- 4. scan ----------------------------------------------------------
  const uint32_t per = (kmax + kThreads - 1) / kThreads;
  const uint32_t k0 = min(kmax, (uint32_t)tid * per), k1 = min(kmax, k0 + per);
  long long cut_t = 0, vol_t = 0;
  for (uint32_t k = k0; k < k1; ++k) {
    cut_t += (int32_t)ord[k];
    vol_t += dgs[k];
  }
  const long long cut_i = warp_prefix_incl(cut_t, lane), vol_i = warp_prefix_incl(vol_t, lane);
  if (lane == 31) {
    s_w64[0][warp] = (unsigned long long)cut_i;
    s_w64[1][warp] = (unsigned long long)vol_i;
  }
  __syncthreads();
  long long cut = cut_i - cut_t, vol = vol_i - vol_t;
  for (int w = 0; w < warp; ++w) {
    cut += (long long)s_w64[0][w];
    vol += (long long)s_w64[1][w];
  }
  const long long vol_all = (long long)a.m;
  double *prow_phi = a.phi ? a.phi + q * a.top : nullptr;
  for (uint32_t k = k0; k < k1; ++k) {
    cut += (int32_t)ord[k];
    vol += dgs[k];
    const long long rest = vol_all - vol;
    const long long den = vol < rest ? vol : rest;
    const double phi = den > 0 ? (double)cut / (double)den : 1.0;
    if (prow_phi) prow_phi[k] = phi;
    if (a.ncp) atomicMin(a.ncp + k, dbl_enc(phi));
  }
  for (uint32_t k = kmax + tid; k < T; k += kThreads) {
    if (orow) orow[k] = -1;
    if (prow_phi) prow_phi[k] = __longlong_as_double(0x7FF8000000000000ll);  // NaN: no such prefix
  }
  if (tid == 0 && a.count) a.count[q] = (int32_t)kmax;
}

// profile: accumulate ? encode the caller's values : start from +inf (encoded)
__global__ void ncp_profile_begin(unsigned long long *ncp, int32_t top, int accumulate) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= top) return;
  const double x = accumulate ? __longlong_as_double((long long)ncp[i]) : __longlong_as_double(0x7FF0000000000000ll);
  ncp[i] = dbl_enc(x);
}

__global__ void ncp_profile_end(unsigned long long *ncp, int32_t top) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < top) ncp[i] = (unsigned long long)__double_as_longlong(dbl_dec(ncp[i]));
}

// out-degree per original id: deg[orig[u]] = rp[u + 1] - rp[u]
__global__ void degree_table(const uint32_t *rp, const int32_t *orig, int64_t n, uint32_t *deg) {
  for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < n; u += (int64_t)gridDim.x * blockDim.x) {
    const int64_t v = orig ? orig[u] : u;
    deg[v] = rp[u + 1] - rp[u];
  }
}

bool aligned(const void *p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

}  // namespace
}  // namespace fg

using namespace fg;

extern "C" fg_status fg_ncp_sweep(fg_graph *g, const float *p, int32_t nq, int32_t top, int32_t *order_out,
                                  double *phi_out, int32_t *count_out, double *ncp_out, int32_t accumulate,
                                  void *stream_v) {
  if (!g) return fail(FG_ERR_INVALID_ARG, "graph is NULL");
  if (!p) return fail(FG_ERR_INVALID_ARG, "p is NULL");
  if (nq <= 0) return fail(FG_ERR_INVALID_ARG, "nq must be > 0 (got %d)", nq);
  if (top < 1 || top > FG_NCP_MAX_TOP)
    return fail(FG_ERR_INVALID_ARG, "top must be in [1, %d] (got %d)", FG_NCP_MAX_TOP, top);
  if (!order_out && !phi_out && !count_out && !ncp_out) return fail(FG_ERR_INVALID_ARG, "no output given");
  if (!aligned(p, 4) || !aligned(order_out, 4) || !aligned(count_out, 4) || !aligned(phi_out, 8) ||
      !aligned(ncp_out, 8))
    return fail(FG_ERR_INVALID_ARG, "misaligned pointer");
  int dev = -1;
  CUDA_TRY(cudaGetDevice(&dev));
  if (dev != g->device)
    return fail(FG_ERR_INVALID_ARG, "the graph lives on device %d but device %d is current", g->device, dev);
  cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_v);
  const int64_t n = g->n;

  {
    // degree table in original order, built once per graph (the only
    // synchronising step; later calls only read it)
    std::lock_guard<std::mutex> lk(g->mu);
    if (!g->deg.p) {
      static std::once_flag attr_once;
      static cudaError_t attr_err = cudaSuccess;
      std::call_once(attr_once, [] {
        attr_err = cudaFuncSetAttribute(ncp_sweep_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem);
        if (attr_err == cudaSuccess)
          attr_err = cudaFuncSetAttribute(ncp_select_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem);
        if (attr_err == cudaSuccess)
          attr_err = cudaFuncSetAttribute(ncp_merge_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem);
      });
      CUDA_TRY(attr_err);
      DevBuf d;
      CUDA_TRY(d.reserve(sizeof(uint32_t) * (size_t)n));
      const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 152 * 16));
      degree_table<<<blocks, 256, 0, stream>>>(g->dg.rp, g->dg.orig, n, d.as<uint32_t>());
      cudaError_t e = cudaGetLastError();
      if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
      if (e != cudaSuccess) {
        d.release();
        return fail(FG_ERR_CUDA, "degree table: %s", cudaGetErrorString(e));
      }
      g->deg = d;
    }
  }

  NcpArgs a;
  a.p = p;
  a.deg = g->deg.as<uint32_t>();
  a.rp = g->dg.rp;
  a.adj = g->dg.adj;
  a.intl = g->dg.intl;
  a.n = n;
  a.m = g->dg.m;
  a.top = top;
  a.order = order_out;
  a.phi = phi_out;
  a.count = count_out;
  a.ncp = reinterpret_cast<unsigned long long *>(ncp_out);
  if (a.ncp) {
    ncp_profile_begin<<<(top + 255) / 256, 256, 0, stream>>>(a.ncp, top, accumulate ? 1 : 0);
    CUDA_TRY(cudaGetLastError());
  }
  const bool vec = (n % 4 == 0) && aligned(p, 16);
  // Rows are split into `parts` segments when there are too few rows to give
  // every SM two blocks: each segment's block keeps its top keys, and one
  // block per row merges them (the kept set does not depend on the split).
  int sms = 0;
  CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int64_t ntiles = (n + kTile - 1) / kTile;
  int64_t parts = (4ll * sms + nq - 1) / nq;
  parts = std::min<int64_t>(std::min<int64_t>(parts, 16), ntiles / 4);
  if (parts <= 1) {
    ncp_sweep_kernel<<<nq, kThreads, kSmem, stream>>>(a, vec);
    CUDA_TRY(cudaGetLastError());
  } else {
    unsigned long long *scratch = nullptr;
    const size_t bytes = (size_t)nq * (size_t)parts * (size_t)top * sizeof(unsigned long long);
    CUDA_TRY(cudaMallocAsync(reinterpret_cast<void **>(&scratch), bytes, stream));
    ncp_select_kernel<<<(unsigned)(nq * parts), kThreads, kSmem, stream>>>(a, vec, (int)parts, scratch);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) {
      ncp_merge_kernel<<<nq, kThreads, kSmem, stream>>>(a, (int)parts, scratch);
      e = cudaGetLastError();
    }
    cudaFreeAsync(scratch, stream);
    CUDA_TRY(e);
  }
  if (a.ncp) {
    ncp_profile_end<<<(top + 255) / 256, 256, 0, stream>>>(a.ncp, top);
    CUDA_TRY(cudaGetLastError());
  }
  return FG_OK;
}
