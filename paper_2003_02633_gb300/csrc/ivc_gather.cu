// Random-access decompression (the unstructured access of Sec. 1): the
// decoded vectors at an index list, AoS FP32 out.  Kernels of their own file
// so that the streaming kernels' sources stay as profiled.
#include "ivc_decode_poles.cuh"
#include "ivc_internal.h"

namespace ivc {
namespace {

#define GATHER_TABLES(F, MAP)                                      \
  extern __shared__ TabEntry ivc_gather_tab[];                     \
  stage_tables<MAP>(F, ivc_gather_tab);                            \
  const TabEntry *tab_t = ivc_gather_tab;                          \
  const TabEntry *tab_p = ivc_gather_tab + (MAP == MAP_TANH ? 0 : F.nent_t)

// Gather-decompress (random access, the motivation of Sec. 1): xyz[i] =
// decompress(w[idx[i]]) for i < n, AoS output.  Indices outside [0, nw) read
// nothing and give NaN components.  Generic kernel: one index per thread.
template <int MAP>
__global__ void __launch_bounds__(256) k_gather(const __grid_constant__ DevFormat F,
                                                const uint64_t *__restrict__ w, int64_t nw,
                                                const int64_t *__restrict__ idx, int64_t n,
                                                float *xyz) {
  GATHER_TABLES(F, MAP);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const int64_t j = __ldcs(idx + i);
    float3 v = make_float3(__int_as_float(0x7fc00000), __int_as_float(0x7fc00000),
                           __int_as_float(0x7fc00000));
    if ((uint64_t)j < (uint64_t)nw) v = decode_word<MAP>(__ldg(w + j), F, tab_t, tab_p);
    __stcs(xyz + 3 * i, v.x);
    __stcs(xyz + 3 * i + 1, v.y);
    __stcs(xyz + 3 * i + 2, v.z);
  }
}

// Fast-path gather: two indices per thread (16-byte index loads), packed
// decode, the same AoS stores as k_decompress_fast.  Requires a 16-byte aligned
// idx and an 8-byte aligned xyz.
template <class G>
__global__ void __launch_bounds__(256) k_gather_fast(const __grid_constant__ DevFormat F,
                                                     const uint64_t *__restrict__ w, int64_t nw,
                                                     const int64_t *__restrict__ idx, int64_t n,
                                                     float *xyz) {
  GATHER_TABLES(F, G::MAP);
  const int64_t n2 = n >> 1;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const longlong2 *i2 = reinterpret_cast<const longlong2 *>(idx);
  float2 *v2 = reinterpret_cast<float2 *>(xyz);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n2; i += stride) {
    const longlong2 jj = __ldcs(i2 + i);
    const bool ok0 = (uint64_t)jj.x < (uint64_t)nw, ok1 = (uint64_t)jj.y < (uint64_t)nw;
    const uint64_t w0 = ok0 ? __ldg(w + jj.x) : 0ull;
    const uint64_t w1 = ok1 ? __ldg(w + jj.y) : 0ull;
    float2 X, Y, Z;
    fast::decode2_poles<G>(w0, w1, F, tab_t, tab_p, X, Y, Z);
    const float qn = __int_as_float(0x7fc00000);
    if (!ok0) X.x = Y.x = Z.x = qn;
    if (!ok1) X.y = Y.y = Z.y = qn;
    __stcs(v2 + 3 * i, make_float2(X.x, Y.x));
    __stcs(v2 + 3 * i + 1, make_float2(Z.x, X.y));
    __stcs(v2 + 3 * i + 2, make_float2(Y.y, Z.y));
  }
  if ((n & 1) && blockIdx.x == 0 && threadIdx.x == 0) {
    const int64_t i = n - 1;
    const int64_t j = idx[i];
    float3 v = make_float3(__int_as_float(0x7fc00000), __int_as_float(0x7fc00000),
                           __int_as_float(0x7fc00000));
    if ((uint64_t)j < (uint64_t)nw) v = decode_word<G::MAP>(w[j], F, tab_t, tab_p);
    xyz[3 * i] = v.x;
    xyz[3 * i + 1] = v.y;
    xyz[3 * i + 2] = v.z;
  }
}

int sm_count_here() {
  int dev = 0, n = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return 1;
  }
  return n > 0 ? n : 1;
}

// Grid: SMs x resident blocks of 256 threads, capped by the work.
template <typename K>
cudaError_t shape_for(K kernel, size_t smem, int64_t work, int *grid) {
  int occ = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, 256, smem);
  if (e != cudaSuccess) return e;
  if (occ < 1) occ = 1;
  int64_t g = (int64_t)sm_count_here() * occ;
  const int64_t need = (work + 255) / 256;
  if (g > need) g = need;
  *grid = (int)(g < 1 ? 1 : g);
  return cudaSuccess;
}

}  // namespace

cudaError_t launch_gather(int map, const DevFormat &F, const uint64_t *w, int64_t nw,
                          const int64_t *idx, int64_t n, float *xyz, bool pairs,
                          cudaStream_t st) {
  const size_t smem = table_smem_bytes(F, map);
  int grid = 1;
  cudaError_t e;
  if (pairs && fast::fast_geometry(map, F) != 0) {
    auto run = [&](auto g) -> cudaError_t {
      cudaError_t e2 = shape_for(k_gather_fast<decltype(g)>, smem, (n + 1) / 2, &grid);
      if (e2 != cudaSuccess) return e2;
      k_gather_fast<decltype(g)><<<grid, 256, smem, st>>>(F, w, nw, idx, n, xyz);
      return cudaGetLastError();
    };
    if (fast::is_geo<fast::GeoTanh>(F)) return run(fast::GeoTanh{});
    if (fast::is_geo<fast::GeoSplit>(F)) return run(fast::GeoSplit{});
    if (fast::is_geo<fast::GeoL1717>(F)) return run(fast::GeoL1717{});
    if (fast::is_geo<fast::GeoL1617>(F)) return run(fast::GeoL1617{});
    return run(fast::GeoPrimary{});
  }
  switch (map) {
    case MAP_UNIFORM:
      if ((e = shape_for(k_gather<MAP_UNIFORM>, smem, n, &grid)) != cudaSuccess) return e;
      k_gather<MAP_UNIFORM><<<grid, 256, smem, st>>>(F, w, nw, idx, n, xyz);
      break;
    case MAP_TANH:
      if ((e = shape_for(k_gather<MAP_TANH>, smem, n, &grid)) != cudaSuccess) return e;
      k_gather<MAP_TANH><<<grid, 256, smem, st>>>(F, w, nw, idx, n, xyz);
      break;
    default:
      if ((e = shape_for(k_gather<MAP_FRACSPLIT>, smem, n, &grid)) != cudaSuccess) return e;
      k_gather<MAP_FRACSPLIT><<<grid, 256, smem, st>>>(F, w, nw, idx, n, xyz);
      break;
  }
  return cudaGetLastError();
}

}  // namespace ivc
