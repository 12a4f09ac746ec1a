// Internal interface between the C ABI layer (ivc_api.cu) and the kernel
// translation units.  Not part of the public ABI.
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>
#include <vector>

#include "../../include/ivc.h"
#include "ivc_device.cuh"
#include "ivc_fast.cuh"

namespace ivc {

enum KernelKind : int {
  K_COMPRESS = 0,
  K_DECOMPRESS = 1,
  K_ADD = 2,
  K_AXPY = 3,
  K_UPDATE = 4,
  K_BATCH_ADD = 5,
  K_BATCH_AXPY = 6,
  K_ADD_FAST = 7,
  K_AXPY_FAST = 8,
  K_UPDATE_FAST = 9,
  K_BATCH_ADD_FAST = 10,
  K_BATCH_AXPY_FAST = 11,
  K_COMPRESS_FAST = 12,
  K_DECOMPRESS_FAST = 13,
};

struct LaunchShape {
  int block;   // threads per block
  int grid;    // blocks
  int vec2;    // 1: two words per 16-byte access where aligned
  size_t smem; // dynamic shared memory (tables)
};

// One field of a batched launch (device copy of ivc_field).
struct FieldDesc {
  const uint64_t *a;
  const uint64_t *b;
  uint64_t *c;
  int64_t n;
  float alpha;
  float pad;
};

// Device view of a batched plan.
struct PlanDev {
  const FieldDesc *fields;
  const int64_t *tile_start;  // nfields + 1 prefix sums of tiles per field
  unsigned long long *counter;
  int *status;
  int64_t total_tiles;
  int nfields;
  int tile;
};

size_t table_smem_bytes(const DevFormat &F, int map);
// Dynamic shared memory of a kernel kind: tables, plus the per-warp queues of
// deferred exact tests for the fast kernels that encode.
size_t kernel_smem_bytes(const DevFormat &F, int map, int kind, int block);

cudaError_t launch_compress(int map, const DevFormat &F, const float *xyz, int layout, int64_t ld,
                            int64_t n, uint64_t *w, ivc_counts *counts, const LaunchShape &s,
                            cudaStream_t st);
cudaError_t launch_decompress(int map, const DevFormat &F, const uint64_t *w, int64_t n,
                              float *xyz, int layout, int64_t ld, const LaunchShape &s,
                              cudaStream_t st);
// The same with every rounding decision through the exact integer helpers
// (AoS only; validation entry points).
cudaError_t launch_compress_exact(int map, const DevFormat &F, const float *xyz, int64_t n,
                                  uint64_t *w, ivc_counts *counts, const LaunchShape &s,
                                  cudaStream_t st);
cudaError_t launch_decompress_exact(int map, const DevFormat &F, const uint64_t *w, int64_t n,
                                    float *xyz, const LaunchShape &s, cudaStream_t st);
cudaError_t launch_add(int map, const DevFormat &F, const uint64_t *a, const uint64_t *b,
                       uint64_t *c, int64_t n, const LaunchShape &s, cudaStream_t st);
cudaError_t launch_axpy(int map, const DevFormat &F, float alpha, const uint64_t *x, uint64_t *y,
                        int64_t n, const LaunchShape &s, cudaStream_t st);
cudaError_t launch_update(int map, const DevFormat &F, float dt, const uint64_t *v,
                          const uint64_t *f, const float *rho, uint64_t *v_out, uint64_t *m_out,
                          int64_t n, const LaunchShape &s, cudaStream_t st);
// Fast path of the primary layout and of the default fractional split
// (requires fast::fast_geometry(map, F) != 0); two words
// per thread, n >= 0, 16-byte aligned word arrays.
cudaError_t launch_add_fast(const DevFormat &F, const uint64_t *a, const uint64_t *b, uint64_t *c,
                            int64_t n, const LaunchShape &s, cudaStream_t st);
cudaError_t launch_axpy_fast(const DevFormat &F, float alpha, const uint64_t *x, uint64_t *y,
                             int64_t n, const LaunchShape &s, cudaStream_t st);
cudaError_t launch_compress_fast(const DevFormat &F, const float *xyz, int64_t n, uint64_t *w,
                                 ivc_counts *counts, const LaunchShape &s, cudaStream_t st);
cudaError_t launch_decompress_fast(const DevFormat &F, const uint64_t *w, int64_t n, float *xyz,
                                   const LaunchShape &s, cudaStream_t st);
cudaError_t launch_update_fast(const DevFormat &F, float dt, const uint64_t *v, const uint64_t *f,
                               const float *rho, uint64_t *v_out, uint64_t *m_out, int64_t n,
                               const LaunchShape &s, cudaStream_t st);
cudaError_t launch_batched(int map, int op, const DevFormat &F, const PlanDev &P,
                           const LaunchShape &s, cudaStream_t st);
// Gather-decompress; pairs selects the two-per-thread kernel (16-byte aligned
// idx, 8-byte aligned xyz) when the layout has a fast path.  Sizes its grid.
cudaError_t launch_gather(int map, const DevFormat &F, const uint64_t *w, int64_t nw,
                          const int64_t *idx, int64_t n, float *xyz, bool pairs,
                          cudaStream_t st);
cudaError_t launch_tile_scan(const FieldDesc *fields, int nfields, int tile, int64_t *tile_start,
                             cudaStream_t st);

// Divergence of a compressed (or, with f32, an FP32) flux, Algorithm 1; the
// launcher sizes its own grid (SMs x resident blocks, capped by the tiles).
cudaError_t launch_flux_div(int map, bool fast_path, bool f32, const DevFormat &F,
                            const void *src, int64_t ld, int ns, int nv, int64_t ne,
                            const float *D, float *div, int64_t ld_out, cudaStream_t st);

// One flux-reconstruction step (5-9, 11) on compressed rows of format (map, F)
// or, with f32, on FP32 rows; in0..in5 and out in the step's argument order
// of the C ABI.  The launcher sizes its own grid.
struct FrCall {
  int step;
  bool f32;
  int map;
  DevFormat F;
  ivc_fr_basis basis;
  ivc_fr_gas gas;
  int dims[3];
  int64_t ne, ld;
  int nv;
  const void *in0, *in1, *in2, *in3, *in4, *in5;
  void *out;
};
cudaError_t launch_fr(const FrCall &call, cudaStream_t st);

// The same divergence on the tensor cores (tcgen05, TF32 head/tail split of
// the FP32 operands); the launcher sizes its own grid (one block per tile of
// 128 elements).
cudaError_t launch_flux_div_tc(int map, bool fast_path, bool f32, const DevFormat &F,
                               const void *src, int64_t ld, int ns, int nv, int64_t ne,
                               const float *D, float *div, int64_t ld_out, cudaStream_t st);
cudaError_t flux_div_tc_status(int *status);

// Reads and clears the flux-divergence kernels' device status word (1: a
// bounded wait between the decoding and the accumulating warps ran out).
cudaError_t flux_div_status(int *status);
// Bound (clock cycles) of every wait of the CUDA-core flux-divergence kernel
// launched from now on; <= 0 restores the default (about a second).
void set_flux_div_wait_limit(long long cycles);

// Resident blocks per SM of a kernel at a block size (0 if it cannot run).
int occupancy(int map, int kind, int block, size_t smem);

// Format fields without table pointers (host only, no device work).
ivc_status format_fields(const ivc_format *f, DevFormat *F, int *map_out);

// Host copies of the folded head tables of a uniform or fractional-split
// format (theta grid, then phi grid: F.nent_t + F.nent_p entries), built by
// the same code as the tables the library caches on the device.
void host_uniform_tables(const DevFormat &F, std::vector<TabEntry> &out);

// Launch shape: block size from cfg (default 256), grid = SMs x resident
// blocks (capped by the work), tables in dynamic shared memory.
LaunchShape default_shape(int map, int kind, const DevFormat &F, int64_t n, int vec2,
                          const ivc_launch_config *cfg);

}  // namespace ivc
