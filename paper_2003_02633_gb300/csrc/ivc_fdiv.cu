// Divergence of a compressed flux: Algorithm 1 (Sec. 4; Table fr_nse, step
// 10).  For each element and solution point k:
//     div(k, p) = sum_j sum_c D[c ns + j][k] X(j, p)_c,   X = decompress(F).
//
// GB300 layout of the work: a block owns a tile of 64 elements and all ns
// output points.  Solution points j are taken in chunks of 8: the block first
// decodes the chunk's words (8 points x nvars rows x 64 elements, coalesced
// along the element index) into shared memory as FP32, then every thread
// accumulates a 4 (points k) x nvars x 4 (elements) block of the output from
// the chunk with FP32 FMAs, reading D (staged once per block) and the decoded
// flux from shared memory.  The contraction has K = 3 ns = 192 terms per
// output for hex elements of degree 3; it runs on the FP32 pipes because its
// operands carry 24-bit significands and the result is compared with an FP32
// summation bound (a TF32 or BF16 tensor-core product would round the decoded
// flux to 11 or 8 bits).
#include "ivc_internal.h"

namespace ivc {
namespace {

constexpr int kTE = 64;       // elements per tile
constexpr int kJC = 8;        // solution points per chunk
constexpr int kMaxNs = 64;
constexpr int kMaxNv = 5;
constexpr int kThreads = 256;

enum : int { FD_GENERIC = 0, FD_FAST = 1, FD_F32 = 2 };

__host__ __device__ constexpr int pad4(int v) { return (v + 3) & ~3; }

// Shared memory: [tables][D: 3 ns x pad4(ns)][X: kJC x nvars x 3 x kTE]
template <int MODE, int MAP>
__global__ void __launch_bounds__(kThreads, 2)
    k_flux_div(const __grid_constant__ DevFormat F, const void *__restrict__ src, int64_t ld,
               int ns, int nv, int64_t ne, const float *__restrict__ D, float *__restrict__ div,
               int64_t ld_out) {
  extern __shared__ __align__(16) unsigned char fd_smem[];
  TabEntry *tabs = reinterpret_cast<TabEntry *>(fd_smem);
  const int ntab = (MODE == FD_F32 || MAP == MAP_TANH) ? 0 : F.nent_t + F.nent_p;
  if (ntab > 0) stage_tables<MAP>(F, tabs);
  const TabEntry *tab_t = tabs;
  const TabEntry *tab_p = tabs + (MAP == MAP_TANH ? 0 : F.nent_t);
  const int nsp = pad4(ns);
  float *Ds = reinterpret_cast<float *>(fd_smem + (size_t)ntab * sizeof(TabEntry));
  float *Xs = Ds + 3 * ns * nsp;
  // D once per block, rows padded to a multiple of 4 columns
  for (int i = threadIdx.x; i < 3 * ns * nsp; i += kThreads) {
    const int r = i / nsp, k = i - r * nsp;
    Ds[i] = k < ns ? D[(int64_t)r * ns + k] : 0.0f;
  }
  __syncthreads();

  const int eg = threadIdx.x & 15;   // elements 4 eg .. 4 eg + 3 of the tile
  const int kg = threadIdx.x >> 4;   // points 4 kg .. 4 kg + 3
  const bool kact = 4 * kg < nsp;
  const int64_t ntiles = (ne + kTE - 1) / kTE;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t e0 = tile * kTE;
    float acc[4][kMaxNv][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int p = 0; p < kMaxNv; ++p)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][p][b] = 0.0f;

    for (int j0 = 0; j0 < ns; j0 += kJC) {
      const int jn = min(kJC, ns - j0);
      __syncthreads();  // the previous chunk's readers are done with Xs
      // decode: jn x nv rows x 64 elements, two adjacent elements per item
      const int items = jn * nv * (kTE / 2);
      for (int q = threadIdx.x; q < items; q += kThreads) {
        const int e2 = q & (kTE / 2 - 1);
        const int r = q / (kTE / 2);
        const int jj = r / nv, p = r - jj * nv;
        const int64_t e = e0 + 2 * e2;
        float2 vx, vy, vz;
        if (MODE == FD_F32) {
          const float *Fr = static_cast<const float *>(src);
          float v[3][2];
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            const int64_t base = (((int64_t)c * ns + j0 + jj) * nv + p) * ld + e;
            v[c][0] = e < ne ? __ldcs(Fr + base) : 0.0f;
            v[c][1] = e + 1 < ne ? __ldcs(Fr + base + 1) : 0.0f;
          }
          vx = make_float2(v[0][0], v[0][1]);
          vy = make_float2(v[1][0], v[1][1]);
          vz = make_float2(v[2][0], v[2][1]);
        } else {
          const uint64_t *W = static_cast<const uint64_t *>(src);
          const int64_t base = ((int64_t)(j0 + jj) * nv + p) * ld + e;
          const uint64_t w0 = e < ne ? __ldcs(W + base) : 0ull;
          const uint64_t w1 = e + 1 < ne ? __ldcs(W + base + 1) : 0ull;
          if (MODE == FD_FAST) {
            fast::decode2_full(w0, w1, F, tab_t, tab_p, vx, vy, vz);
          } else {
            const float3 a = decode_word<MAP>(w0, F, tab_t, tab_p);
            const float3 b = decode_word<MAP>(w1, F, tab_t, tab_p);
            vx = make_float2(a.x, b.x);
            vy = make_float2(a.y, b.y);
            vz = make_float2(a.z, b.z);
          }
        }
        float *xr = Xs + ((jj * kMaxNv + p) * 3) * kTE + 2 * e2;
        *reinterpret_cast<float2 *>(xr) = vx;
        *reinterpret_cast<float2 *>(xr + kTE) = vy;
        *reinterpret_cast<float2 *>(xr + 2 * kTE) = vz;
      }
      __syncthreads();
      if (kact) {
        for (int jj = 0; jj < jn; ++jj) {
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            const float4 d =
                *reinterpret_cast<const float4 *>(Ds + (c * ns + j0 + jj) * nsp + 4 * kg);
            const float dk[4] = {d.x, d.y, d.z, d.w};
#pragma unroll
            for (int p = 0; p < kMaxNv; ++p) {
              if (p < nv) {
                const float4 x = *reinterpret_cast<const float4 *>(
                    Xs + ((jj * kMaxNv + p) * 3 + c) * kTE + 4 * eg);
                const float xe[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
                for (int a = 0; a < 4; ++a)
#pragma unroll
                  for (int b = 0; b < 4; ++b) acc[a][p][b] = fmaf(dk[a], xe[b], acc[a][p][b]);
              }
            }
          }
        }
      }
    }
    // epilogue: points 4 kg + a < ns, elements e0 + 4 eg + b < ne
    if (kact) {
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        const int k = 4 * kg + a;
        if (k >= ns) continue;
#pragma unroll
        for (int p = 0; p < kMaxNv; ++p) {
          if (p >= nv) continue;
          float *o = div + ((int64_t)k * nv + p) * ld_out + e0 + 4 * eg;
          const int64_t e = e0 + 4 * eg;
          if (e + 3 < ne && (reinterpret_cast<uintptr_t>(o) & 15u) == 0) {
            __stcs(reinterpret_cast<float4 *>(o),
                   make_float4(acc[a][p][0], acc[a][p][1], acc[a][p][2], acc[a][p][3]));
          } else {
#pragma unroll
            for (int b = 0; b < 4; ++b)
              if (e + b < ne) o[b] = acc[a][p][b];
          }
        }
      }
    }
  }
}

template <int MODE, int MAP>
cudaError_t launch_one(const DevFormat &F, const void *src, int64_t ld, int ns, int nv,
                       int64_t ne, const float *D, float *div, int64_t ld_out, cudaStream_t st) {
  const int ntab = (MODE == FD_F32 || MAP == MAP_TANH) ? 0 : F.nent_t + F.nent_p;
  const size_t smem = (size_t)ntab * sizeof(TabEntry) +
                      (size_t)(3 * ns * pad4(ns)) * sizeof(float) +
                      (size_t)kJC * kMaxNv * 3 * kTE * sizeof(float);
  const void *k = (const void *)k_flux_div<MODE, MAP>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 1, occ = 1;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
    return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, kThreads, smem)) != cudaSuccess)
    return e;
  if (occ < 1) return cudaErrorInvalidConfiguration;
  const int64_t ntiles = (ne + kTE - 1) / kTE;
  int64_t grid = (int64_t)sms * occ;
  if (grid > ntiles) grid = ntiles;
  k_flux_div<MODE, MAP><<<(int)grid, kThreads, smem, st>>>(F, src, ld, ns, nv, ne, D, div,
                                                            ld_out);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_flux_div(int map, bool fast_path, bool f32, const DevFormat &F,
                            const void *src, int64_t ld, int ns, int nv, int64_t ne,
                            const float *D, float *div, int64_t ld_out, cudaStream_t st) {
  if (ns < 1 || ns > kMaxNs || nv < 1 || nv > kMaxNv) return cudaErrorInvalidValue;
  if (f32) return launch_one<FD_F32, MAP_UNIFORM>(F, src, ld, ns, nv, ne, D, div, ld_out, st);
  if (fast_path)
    return launch_one<FD_FAST, MAP_UNIFORM>(F, src, ld, ns, nv, ne, D, div, ld_out, st);
  switch (map) {
    case MAP_UNIFORM:
      return launch_one<FD_GENERIC, MAP_UNIFORM>(F, src, ld, ns, nv, ne, D, div, ld_out, st);
    case MAP_TANH:
      return launch_one<FD_GENERIC, MAP_TANH>(F, src, ld, ns, nv, ne, D, div, ld_out, st);
    default:
      return launch_one<FD_GENERIC, MAP_FRACSPLIT>(F, src, ld, ns, nv, ne, D, div, ld_out, st);
  }
}

}  // namespace ivc
