// ivc_add_noalloc: the compressed add without any device allocation.
//
// Who needs it: code that must not call cudaMalloc on its path, for example a
// caller inside a framework whose caching allocator already owns the device
// memory, a latency-critical loop where cudaMalloc's implicit device-wide
// synchronisation is not acceptable, or a teardown / error path where an
// allocation may fail.  ivc_add builds and caches its trigonometric tables in
// cudaMalloc'd memory on first use of a format; this entry point keeps them in
// a fixed file-scope device array instead.
//
// The array (kNoAllocEntries table entries, 32 KiB) is part of the library
// image, so every GPU that loads the library holds it until process exit.
// Host code cannot use the array's name as a device address; the device
// address is looked up once per device with cudaGetSymbolAddress, on the
// first call made with that device current.  All calls share the array and it
// keeps the last call's contents: a call whose format differs from the one the
// array holds on that device first rewrites the tables (an asynchronous copy of
// host-built tables, the same values ivc_add caches, on the call's stream) and
// records an event after the copy; every call makes its stream wait for the
// latest such event before its kernel, so a call on another stream or host
// thread never reads tables that are still being written.  Calls that overlap
// on the GPU and use different formats still race on the array.  A call that
// would rewrite the tables, or the first call on a device, is refused while its
// stream is capturing (IVC_ERR_UNSUPPORTED): a captured call reads whatever the
// array holds when the graph runs, which a later call with another format
// rewrites.
#include <mutex>
#include <vector>

#include "ivc_internal.h"

namespace {

constexpr int kNoAllocEntries = 2048;  // theta + phi head-table entries
constexpr int kMaxDevices = 64;

static __device__ __align__(256) ivc::TabEntry g_noalloc_tab[kNoAllocEntries];

struct DeviceSlot {
  ivc::TabEntry *tab = nullptr;       // device address of g_noalloc_tab
  cudaEvent_t filled = nullptr;       // recorded after the latest table copy
  bool has_fill = false;              // filled has been recorded at least once
  int Dt = -1, Dp = -1, st = -1, sp = -1;  // format whose tables the array holds
};

std::mutex g_slot_mu;
DeviceSlot g_slots[kMaxDevices];

bool aligned(const void *p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

}  // namespace

extern "C" ivc_status ivc_add_noalloc(const ivc_format *fmt, const uint64_t *a, const uint64_t *b,
                                      uint64_t *c, int64_t n, ivc_stream_t stream) {
  using namespace ivc;
  if (n < 0) return IVC_ERR_ARG;
  DevFormat F;
  int map = 0;
  ivc_status st = format_fields(fmt, &F, &map);
  if (st != IVC_OK) return st;
  if (map == IVC_MAP_TANH) return IVC_ERR_UNSUPPORTED;  // per-code tables exceed the array
  if (F.nent_t + F.nent_p > kNoAllocEntries) return IVC_ERR_NOMEM;
  if (n == 0) return IVC_OK;
  if (!a || !b || !c) return IVC_ERR_ARG;
  if (!aligned(a, 8) || !aligned(b, 8) || !aligned(c, 8)) return IVC_ERR_ALIGN;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return IVC_ERR_CUDA;
  }
  if (dev < 0 || dev >= kMaxDevices) return IVC_ERR_UNSUPPORTED;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(stream, &cap) != cudaSuccess) {
    cudaGetLastError();
    return IVC_ERR_CUDA;
  }
  const bool capturing = cap != cudaStreamCaptureStatusNone;
  {
    std::lock_guard<std::mutex> lk(g_slot_mu);
    DeviceSlot &slot = g_slots[dev];
    if (slot.tab == nullptr) {
      if (capturing) return IVC_ERR_UNSUPPORTED;
      void *p = nullptr;
      if (cudaGetSymbolAddress(&p, g_noalloc_tab) != cudaSuccess || p == nullptr) {
        cudaGetLastError();
        return IVC_ERR_CUDA;
      }
      if (cudaEventCreateWithFlags(&slot.filled, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        return IVC_ERR_CUDA;
      }
      slot.tab = static_cast<TabEntry *>(p);
    }
    if (slot.Dt != F.Dt || slot.Dp != F.Dp || slot.st != F.st || slot.sp != F.sp) {
      if (capturing) return IVC_ERR_UNSUPPORTED;
      // the same host tables ivc_add caches; the copy from pageable memory is
      // staged before this call returns, so the vector may go out of scope
      std::vector<TabEntry> host;
      host.reserve((size_t)(F.nent_t + F.nent_p));
      host_uniform_tables(F, host);
      if (host.size() != (size_t)(F.nent_t + F.nent_p)) return IVC_ERR_FORMAT;
      if (cudaMemcpyToSymbolAsync(g_noalloc_tab, host.data(), host.size() * sizeof(TabEntry), 0,
                                  cudaMemcpyHostToDevice, stream) != cudaSuccess ||
          cudaEventRecord(slot.filled, stream) != cudaSuccess) {
        cudaGetLastError();
        slot.Dt = slot.Dp = slot.st = slot.sp = -1;  // contents unknown: refill next time
        return IVC_ERR_CUDA;
      }
      slot.has_fill = true;
      slot.Dt = F.Dt;
      slot.Dp = F.Dp;
      slot.st = F.st;
      slot.sp = F.sp;
    } else if (!capturing && slot.has_fill) {
      // the tables may still be in flight on the stream that wrote them
      if (cudaStreamWaitEvent(stream, slot.filled, 0) != cudaSuccess) {
        cudaGetLastError();
        return IVC_ERR_CUDA;
      }
    }
    F.tab = slot.tab;
  }
  const bool vec2 = aligned(a, 16) && aligned(b, 16) && aligned(c, 16);
  cudaError_t e;
  if (vec2 && fast::fast_geometry(map, F) != 0) {
    e = launch_add_fast(F, a, b, c, n, default_shape(map, K_ADD_FAST, F, n, 1, nullptr), stream);
  } else {
    e = launch_add(map, F, a, b, c, n, default_shape(map, K_ADD, F, n, vec2 ? 1 : 0, nullptr),
                   stream);
  }
  return e == cudaSuccess ? IVC_OK : IVC_ERR_CUDA;
}
