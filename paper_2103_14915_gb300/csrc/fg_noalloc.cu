// SSSP batch that allocates no memory: the plain per-query kernel launched on
// scratch that is compiled into the library instead of scratch taken from the
// graph's workspace (which fg_sssp_batch grows with cudaMalloc on demand).
//
// Who cannot allocate: a caller whose device memory is fixed up front by
// another component (a serving process that hands all free HBM to its own
// pool), and a caller that keeps independent work running on other streams
// and cannot accept the implicit device-wide synchronisation of cudaFree when
// a workspace is regrown. Such callers still get exact distances for graphs of
// up to FG_NOALLOC_MAX_VERTICES vertices.
#include <cstdio>
#include <mutex>

#include "fg_internal.h"

namespace fg {
namespace {

constexpr size_t kAlign = 256;
constexpr size_t kMaxN = (size_t)FG_NOALLOC_MAX_VERTICES;
constexpr size_t kCtrlBytes = (sizeof(Ctrl) + kAlign - 1) / kAlign * kAlign;
constexpr size_t kSizesBytes = kAlign;  // three frontier sizes
constexpr size_t kRowBytes = 4 * kMaxN;  // one uint32 per vertex
// Layout: [Ctrl][sizes][dist][stamp][frontier 0][frontier 1]
constexpr size_t kScratchBytes = kCtrlBytes + kSizesBytes + 4 * kRowBytes;
static_assert(kRowBytes % kAlign == 0, "scratch rows must keep 256-byte alignment");
static_assert(kScratchBytes == 16u * 1024u * 1024u + 2u * kAlign, "scratch is 16 MiB of rows plus two headers");

// Zero when the module is loaded. Only the control block must be zero when a
// kernel starts; every call clears it before its first launch. The kernel
// itself writes dist, stamp and the sizes before reading them, and reads only
// frontier entries it wrote in the same launch.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;

struct DeviceSetup {
  bool done = false;
  unsigned char *base = nullptr;  // device address of g_noalloc_scratch on this device
  int blocks = 0, threads = 0;    // cooperative grid of the plain kernel
};

std::mutex g_setup_mu;
DeviceSetup g_setup[kMaxDevices];

// Formats into the caller's stack: calls on different devices may fail at the
// same time, and each thread's fg_last_error() must carry its own message.
fg_status fail_msg(fg_status s, const char *fmt, long long a, long long b) {
  char msg[256];
  std::snprintf(msg, sizeof(msg), fmt, a, b);
  return report_error(s, msg);
}

// Set-up of one device (that device current): look up the scratch's device
// address and the plain kernel's cooperative grid. With lazy module loading
// (CUDA's default) the lookup is what loads the module and places the scratch
// array in device memory, and the occupancy query loads the plain kernel; a
// memset of the control block brings up the runtime's memset path. All of it
// happens here, once, so that later calls on the device take no memory and
// load nothing. Retried on failure.
fg_status setup_device(int dev, const DeviceSetup **out) {
  std::lock_guard<std::mutex> lk(g_setup_mu);
  DeviceSetup &s = g_setup[dev];
  if (!s.done) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return report_error(FG_ERR_CUDA, cudaGetErrorString(e));
    if (reinterpret_cast<uintptr_t>(p) % kAlign != 0)
      return report_error(FG_ERR_CUDA, "no-allocation scratch is not 256-byte aligned");
    int blocks = 0, threads = 0;
    e = plain_grid_size(&blocks, &threads);
    if (e != cudaSuccess) return report_error(FG_ERR_CUDA, cudaGetErrorString(e));
    e = cudaMemset(p, 0, sizeof(Ctrl));
    if (e != cudaSuccess) return report_error(FG_ERR_CUDA, cudaGetErrorString(e));
    s.base = static_cast<unsigned char *>(p);
    s.blocks = blocks;
    s.threads = threads;
    s.done = true;
  }
  if (out) *out = &s;
  return FG_OK;
}

}  // namespace

// Called by fg_graph_create on the graph's device (current), so that the
// scratch is in place before the caller's own pool takes the free memory.
// A failure here is not an error of graph creation: the first
// fg_sssp_batch_noalloc call on the device retries and reports it.
void noalloc_prepare(int dev) {
  if (dev < 0 || dev >= kMaxDevices) return;
  if (setup_device(dev, nullptr) != FG_OK) {
    (void)cudaGetLastError();
    report_error(FG_OK, "");
  }
}

}  // namespace fg

using namespace fg;

extern "C" fg_status fg_sssp_batch_noalloc(const fg_graph *g, const int32_t *src, int32_t nq, uint32_t *dist_out,
                                           void *stream_v) {
  if (!g) return report_error(FG_ERR_INVALID_ARG, "graph is NULL");
  if (nq <= 0) return report_error(FG_ERR_INVALID_ARG, "nq must be > 0");
  if (!src || !dist_out) return report_error(FG_ERR_INVALID_ARG, "src or dist_out is NULL");
  if ((reinterpret_cast<uintptr_t>(src) & 3u) || (reinterpret_cast<uintptr_t>(dist_out) & 3u))
    return report_error(FG_ERR_INVALID_ARG, "misaligned pointer");
  DevGraph dg;
  int gdev = 0;
  graph_device_view(g, &dg, &gdev);
  if ((size_t)dg.n > kMaxN)
    return fail_msg(FG_ERR_UNSUPPORTED,
                    "graph has %lld vertices; the fixed scratch of fg_sssp_batch_noalloc holds at most %lld",
                    (long long)dg.n, (long long)kMaxN);
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return report_error(FG_ERR_CUDA, cudaGetErrorString(e));
  if (dev != gdev)
    return fail_msg(FG_ERR_INVALID_ARG, "the graph lives on device %lld but device %lld is current",
                    (long long)gdev, (long long)dev);
  if (dev < 0 || dev >= kMaxDevices) return report_error(FG_ERR_UNSUPPORTED, "device ordinal beyond 63");
  const DeviceSetup *s = nullptr;
  fg_status st = setup_device(dev, &s);
  if (st != FG_OK) return st;

  cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_v);
  Ctrl *ctrl = reinterpret_cast<Ctrl *>(s->base);
  uint32_t *sizes = reinterpret_cast<uint32_t *>(s->base + kCtrlBytes);
  uint32_t *rows = reinterpret_cast<uint32_t *>(s->base + kCtrlBytes + kSizesBytes);
  e = cudaMemsetAsync(ctrl, 0, sizeof(Ctrl), stream);
  if (e != cudaSuccess) return report_error(FG_ERR_CUDA, cudaGetErrorString(e));
  for (int32_t q = 0; q < nq; ++q) {
    PlainArgs a;
    a.g = dg;
    a.qtype = Q_SSSP;
    a.q = q;
    a.nq = nq;
    a.src = src;
    a.out_u32 = dist_out + (size_t)q * (size_t)dg.n;
    a.dist = rows;
    a.stamp = rows + kMaxN;
    a.front[0] = rows + 2 * kMaxN;
    a.front[1] = rows + 3 * kMaxN;
    a.sizes = sizes;
    a.max_rounds = 1000000u;
    a.watchdog_ns = 30ull * 1000000000ull;
    a.ctrl = ctrl;
    e = launch_plain(a, s->blocks, s->threads, stream);
    if (e != cudaSuccess) return report_error(FG_ERR_CUDA, cudaGetErrorString(e));
  }
  // Device-side errors come back through the control block. A copy into
  // pageable host memory returns only once it is complete.
  Ctrl h;
  e = cudaMemcpyAsync(&h, ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
  if (e != cudaSuccess) return report_error(FG_ERR_CUDA, cudaGetErrorString(e));
  switch (h.status) {
    case 0: return FG_OK;
    case FG_ERR_INVALID_ARG: return report_error(FG_ERR_INVALID_ARG, "device reported: source id out of range");
    case FG_ERR_OVERFLOW: return report_error(FG_ERR_OVERFLOW, "device reported: distance reached 2^32 - 1");
    case FG_ERR_TIMEOUT: return report_error(FG_ERR_TIMEOUT, "device reported: watchdog timeout");
    default: return report_error((fg_status)h.status, "device reported an error");
  }
}
