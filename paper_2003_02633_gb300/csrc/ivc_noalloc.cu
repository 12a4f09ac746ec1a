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
// array holds on that device first rewrites the tables (a small kernel on the
// same stream).  Calls that overlap on the GPU (other streams, other host
// threads) and use different formats race on the array.
#include <mutex>

#include "ivc_internal.h"

namespace {

constexpr int kNoAllocEntries = 2048;  // theta + phi head-table entries
constexpr int kMaxDevices = 64;

static __device__ __align__(256) ivc::TabEntry g_noalloc_tab[kNoAllocEntries];

struct DeviceSlot {
  ivc::TabEntry *tab = nullptr;  // device address of g_noalloc_tab
  int Dt = -1, Dp = -1, st = -1, sp = -1;  // format whose tables the array holds
};

std::mutex g_slot_mu;
DeviceSlot g_slots[kMaxDevices];

// Head tables of the two folded grids (entries at b = i 2^s, angle
// pi b / (2D)), in FP64 then split to head + tail FP32.
__global__ void k_fill_tables(ivc::TabEntry *tab, int Dt, int st, int nt, int Dp, int sp, int np) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nt + np) return;
  const bool is_t = i < nt;
  const int j = is_t ? i : i - nt;
  const int D = is_t ? Dt : Dp;
  const int s = is_t ? st : sp;
  double sv = 0.0, cv = 1.0;
  if (j > 0) sincospi((double)((long long)j << s) / (2.0 * (double)D), &sv, &cv);
  ivc::TabEntry e;
  e.ch = (float)cv;
  e.cl = (float)(cv - (double)e.ch);
  e.sh = (float)sv;
  e.sl = (float)(sv - (double)e.sh);
  tab[i] = e;
}

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
  {
    std::lock_guard<std::mutex> lk(g_slot_mu);
    DeviceSlot &slot = g_slots[dev];
    if (slot.tab == nullptr) {
      void *p = nullptr;
      if (cudaGetSymbolAddress(&p, g_noalloc_tab) != cudaSuccess || p == nullptr) {
        cudaGetLastError();
        return IVC_ERR_CUDA;
      }
      slot.tab = static_cast<TabEntry *>(p);
    }
    if (slot.Dt != F.Dt || slot.Dp != F.Dp || slot.st != F.st || slot.sp != F.sp) {
      const int total = F.nent_t + F.nent_p;
      k_fill_tables<<<(total + 255) / 256, 256, 0, stream>>>(slot.tab, F.Dt, F.st, F.nent_t,
                                                              F.Dp, F.sp, F.nent_p);
      if (cudaGetLastError() != cudaSuccess) return IVC_ERR_CUDA;
      slot.Dt = F.Dt;
      slot.Dp = F.Dp;
      slot.st = F.st;
      slot.sp = F.sp;
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
