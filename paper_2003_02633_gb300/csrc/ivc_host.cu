// ivc_add_host: the compressed add (Sec. 5) of words that live in host
// memory.  Page-locked (pinned) host words are read and written by the kernel
// itself over the host link, on the caller's stream (zero-copy: measured
// faster than staging on GB300, whose device-to-host copies are the slower
// direction).  Other host memory streams through device staging buffers
// carved from the caller's workspace, in chunks, on three streams of the
// library's own, so that the host-to-device copies of one chunk, the kernel
// of the previous one and the device-to-host copy of the one before overlap.
// Ordering with the caller's stream: the chunks start after the work already
// queued on it, and the caller's stream waits for the last chunk.
#include <mutex>

#include "ivc_internal.h"

namespace {

constexpr int kSlots = 3;
constexpr int kMaxDevices = 64;

struct HostPipe {
  bool ready = false;
  cudaStream_t s[kSlots] = {};
  cudaEvent_t done[kSlots] = {};
  cudaEvent_t start = nullptr;
};

std::mutex g_pipe_mu;
HostPipe g_pipes[kMaxDevices];

bool aligned(const void *p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

// True for page-locked host memory the device can address directly.
bool pinned(const void *p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeHost && at.devicePointer == p;
}

// Streams and events of a device, created on first use and kept until exit.
cudaError_t pipe_of(int dev, HostPipe **out) {
  HostPipe &p = g_pipes[dev];
  if (!p.ready) {
    for (int i = 0; i < kSlots; ++i) {
      cudaError_t e = cudaStreamCreateWithFlags(&p.s[i], cudaStreamNonBlocking);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p.done[i], cudaEventDisableTiming);
      if (e != cudaSuccess) return e;
    }
    cudaError_t e = cudaEventCreateWithFlags(&p.start, cudaEventDisableTiming);
    if (e != cudaSuccess) return e;
    p.ready = true;
  }
  *out = &p;
  return cudaSuccess;
}

}  // namespace

extern "C" ivc_status ivc_add_host(const ivc_format *fmt, const uint64_t *a, const uint64_t *b,
                                   uint64_t *c, int64_t n, void *workspace, size_t ws_bytes,
                                   ivc_stream_t stream) {
  using namespace ivc;
  if (n < 0) return IVC_ERR_ARG;
  DevFormat F;
  int map = 0;
  ivc_status st = format_fields(fmt, &F, &map);
  if (st != IVC_OK) return st;
  if (n == 0) return IVC_OK;
  if (!a || !b || !c) return IVC_ERR_ARG;
  if (!aligned(a, 8) || !aligned(b, 8) || !aligned(c, 8)) return IVC_ERR_ALIGN;
  if (pinned(a) && pinned(b) && pinned(c)) return ivc_add(fmt, a, b, c, n, stream);
  if (!workspace) return IVC_ERR_ARG;
  if (!aligned(workspace, 16)) return IVC_ERR_ALIGN;
  // three slots of (a, b, c) chunks; an even chunk keeps every slot 16-byte aligned
  const int64_t chunk = (int64_t)(ws_bytes / (kSlots * 3 * sizeof(uint64_t))) & ~(int64_t)1;
  if (chunk < 2) return IVC_ERR_NOMEM;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return IVC_ERR_CUDA;
  }
  if (dev < 0 || dev >= kMaxDevices) return IVC_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lk(g_pipe_mu);
  HostPipe *p = nullptr;
  cudaError_t e = pipe_of(dev, &p);
  if (e == cudaSuccess) e = cudaEventRecord(p->start, stream);
  for (int i = 0; e == cudaSuccess && i < kSlots; ++i) e = cudaStreamWaitEvent(p->s[i], p->start, 0);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return IVC_ERR_CUDA;
  }
  uint64_t *ws = static_cast<uint64_t *>(workspace);
  int64_t k = 0;
  for (int64_t off = 0; off < n; off += chunk, ++k) {
    const int slot = (int)(k % kSlots);
    const int64_t m = (n - off < chunk) ? n - off : chunk;
    uint64_t *da = ws + (size_t)slot * 3 * chunk;
    uint64_t *db = da + chunk;
    uint64_t *dc = db + chunk;
    cudaStream_t s = p->s[slot];
    const size_t bytes = (size_t)m * sizeof(uint64_t);
    e = cudaMemcpyAsync(da, a + off, bytes, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(db, b + off, bytes, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) break;
    st = ivc_add(fmt, da, db, dc, m, s);
    if (st != IVC_OK) return st;
    e = cudaMemcpyAsync(c + off, dc, bytes, cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) break;
  }
  for (int i = 0; e == cudaSuccess && i < kSlots; ++i) {
    e = cudaEventRecord(p->done[i], p->s[i]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(stream, p->done[i], 0);
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    return IVC_ERR_CUDA;
  }
  return IVC_OK;
}
