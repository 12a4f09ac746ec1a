// Uncompressed baselines (FP32 AoS / SoA, FP16 / BF16 AoS) of the paper's
// C = A + B benchmark (Sec. 5) and axpy, the FP32 <-> 16-bit storage
// conversions, and the FP64 error reductions of Eq. (stat) / Sec. 3.
//
// The baselines stream flat arrays with 16-byte vector accesses (float4 or
// 8 x 16-bit) and streaming cache hints; scalar code handles any ragged head
// or tail.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "ivc_internal.h"

namespace {

bool aligned(const void *p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

int sm_count() {
  int dev = 0, n = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return 1;
  }
  return n > 0 ? n : 1;
}

int grid_for(int64_t work, int block, int per_sm) {
  int64_t need = (work + block - 1) / block;
  int64_t cap = (int64_t)sm_count() * per_sm;
  if (need > cap) need = cap;
  return need < 1 ? 1 : (int)need;
}

ivc_status st_of(cudaError_t e) { return e == cudaSuccess ? IVC_OK : IVC_ERR_CUDA; }

// ----------------------------------------------------------------- FP32

// out = a + b (alpha == nullptr semantics via flag) or out = fmaf(alpha, a, b)
// over `count` floats per row; row r at offset r * ld (gridDim.y rows).
template <bool AXPY>
__global__ void __launch_bounds__(256) k_f32(const float *a, const float *b, float *out,
                                             float alpha, int64_t count, int64_t ld, int vec4) {
  const int64_t off = (int64_t)blockIdx.y * ld;
  a += off;
  b += off;
  out += off;
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nth = (int64_t)gridDim.x * blockDim.x;
  if (vec4) {
    const int64_t n4 = count >> 2;
    const float4 *a4 = reinterpret_cast<const float4 *>(a);
    const float4 *b4 = reinterpret_cast<const float4 *>(b);
    float4 *o4 = reinterpret_cast<float4 *>(out);
    for (int64_t i = tid; i < n4; i += nth) {
      const float4 x = __ldcs(a4 + i), y = __ldcs(b4 + i);
      float4 r;
      if (AXPY) {
        r = make_float4(fmaf(alpha, x.x, y.x), fmaf(alpha, x.y, y.y), fmaf(alpha, x.z, y.z),
                        fmaf(alpha, x.w, y.w));
      } else {
        r = make_float4(x.x + y.x, x.y + y.y, x.z + y.z, x.w + y.w);
      }
      __stcs(o4 + i, r);
    }
    for (int64_t i = (n4 << 2) + tid; i < count; i += nth) {
      out[i] = AXPY ? fmaf(alpha, a[i], b[i]) : a[i] + b[i];
    }
  } else {
    for (int64_t i = tid; i < count; i += nth) {
      const float x = __ldcs(a + i), y = __ldcs(b + i);
      __stcs(out + i, AXPY ? fmaf(alpha, x, y) : x + y);
    }
  }
}

ivc_status f32_op(bool axpy, ivc_layout layout, float alpha, const float *a, const float *b,
                  float *c, int64_t ld, int64_t n, cudaStream_t st) {
  if (n < 0 || (layout != IVC_AOS && layout != IVC_SOA)) return IVC_ERR_ARG;
  if (layout == IVC_SOA && ld < n) return IVC_ERR_ARG;
  if (n == 0) return IVC_OK;
  if (!a || !b || !c) return IVC_ERR_ARG;
  if (!aligned(a, 4) || !aligned(b, 4) || !aligned(c, 4)) return IVC_ERR_ALIGN;
  const int64_t count = layout == IVC_AOS ? 3 * n : n;
  const int64_t rld = layout == IVC_AOS ? 0 : ld;
  const int rows = layout == IVC_AOS ? 1 : 3;
  const int vec4 = aligned(a, 16) && aligned(b, 16) && aligned(c, 16) &&
                   (layout == IVC_AOS || (ld % 4) == 0);
  dim3 grid(grid_for((vec4 ? count / 4 : count) + 1, 256, 8 / rows > 0 ? 8 / rows : 1), rows);
  if (axpy)
    k_f32<true><<<grid, 256, 0, st>>>(a, b, c, alpha, count, rld, vec4);
  else
    k_f32<false><<<grid, 256, 0, st>>>(a, b, c, alpha, count, rld, vec4);
  return st_of(cudaGetLastError());
}

// FP32 gather (baseline of the gather-decompress): out[i] = src[idx[i]], AoS
// output; source AoS (3 floats at 3 j) or SoA (rows at stride ld).  Indices
// outside [0, nsrc) give NaN components without a read.
template <bool SOA>
__global__ void __launch_bounds__(256) k_f32_gather(const float *__restrict__ src, int64_t ld,
                                                    int64_t nsrc, const int64_t *__restrict__ idx,
                                                    int64_t n, float *out) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const int64_t j = __ldcs(idx + i);
    float x = __int_as_float(0x7fc00000), y = x, z = x;
    if ((uint64_t)j < (uint64_t)nsrc) {
      if (SOA) {
        x = __ldg(src + j);
        y = __ldg(src + ld + j);
        z = __ldg(src + 2 * ld + j);
      } else {
        x = __ldg(src + 3 * j);
        y = __ldg(src + 3 * j + 1);
        z = __ldg(src + 3 * j + 2);
      }
    }
    __stcs(out + 3 * i, x);
    __stcs(out + 3 * i + 1, y);
    __stcs(out + 3 * i + 2, z);
  }
}

// ------------------------------------------------------------ FP16 / BF16

template <int KIND>
__device__ __forceinline__ float h2f(uint16_t v) {
  if (KIND == IVC_F16) return __half2float(__ushort_as_half(v));
  return __bfloat162float(__ushort_as_bfloat16(v));
}

template <int KIND>
__device__ __forceinline__ uint16_t f2h(float v) {
  if (KIND == IVC_F16) return __half_as_ushort(__float2half_rn(v));
  return __bfloat16_as_ushort(__float2bfloat16_rn(v));
}

template <int KIND, bool AXPY>
__device__ __forceinline__ uint32_t op_pair(uint32_t x, uint32_t y, float alpha) {
  const float x0 = h2f<KIND>((uint16_t)(x & 0xffffu)), x1 = h2f<KIND>((uint16_t)(x >> 16));
  const float y0 = h2f<KIND>((uint16_t)(y & 0xffffu)), y1 = h2f<KIND>((uint16_t)(y >> 16));
  const float r0 = AXPY ? fmaf(alpha, x0, y0) : x0 + y0;
  const float r1 = AXPY ? fmaf(alpha, x1, y1) : x1 + y1;
  return (uint32_t)f2h<KIND>(r0) | ((uint32_t)f2h<KIND>(r1) << 16);
}

template <int KIND, bool AXPY>
__global__ void __launch_bounds__(256) k_half(const uint16_t *a, const uint16_t *b, uint16_t *out,
                                              float alpha, int64_t count, int vec) {
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nth = (int64_t)gridDim.x * blockDim.x;
  int64_t done = 0;
  if (vec) {
    const int64_t n8 = count >> 3;
    const uint4 *a4 = reinterpret_cast<const uint4 *>(a);
    const uint4 *b4 = reinterpret_cast<const uint4 *>(b);
    uint4 *o4 = reinterpret_cast<uint4 *>(out);
    for (int64_t i = tid; i < n8; i += nth) {
      const uint4 x = __ldcs(a4 + i), y = __ldcs(b4 + i);
      uint4 r;
      r.x = op_pair<KIND, AXPY>(x.x, y.x, alpha);
      r.y = op_pair<KIND, AXPY>(x.y, y.y, alpha);
      r.z = op_pair<KIND, AXPY>(x.z, y.z, alpha);
      r.w = op_pair<KIND, AXPY>(x.w, y.w, alpha);
      __stcs(o4 + i, r);
    }
    done = n8 << 3;
  }
  for (int64_t i = done + tid; i < count; i += nth) {
    const float x = h2f<KIND>(a[i]), y = h2f<KIND>(b[i]);
    out[i] = f2h<KIND>(AXPY ? fmaf(alpha, x, y) : x + y);
  }
}

ivc_status half_op(bool axpy, ivc_half_kind kind, float alpha, const uint16_t *a,
                   const uint16_t *b, uint16_t *c, int64_t n, cudaStream_t st) {
  if (n < 0 || (kind != IVC_F16 && kind != IVC_BF16)) return IVC_ERR_ARG;
  if (n == 0) return IVC_OK;
  if (!a || !b || !c) return IVC_ERR_ARG;
  if (!aligned(a, 2) || !aligned(b, 2) || !aligned(c, 2)) return IVC_ERR_ALIGN;
  const int64_t count = 3 * n;
  const int vec = aligned(a, 16) && aligned(b, 16) && aligned(c, 16);
  const int grid = grid_for((vec ? count / 8 : count) + 1, 256, 8);
  if (kind == IVC_F16) {
    if (axpy) k_half<IVC_F16, true><<<grid, 256, 0, st>>>(a, b, c, alpha, count, vec);
    else k_half<IVC_F16, false><<<grid, 256, 0, st>>>(a, b, c, alpha, count, vec);
  } else {
    if (axpy) k_half<IVC_BF16, true><<<grid, 256, 0, st>>>(a, b, c, alpha, count, vec);
    else k_half<IVC_BF16, false><<<grid, 256, 0, st>>>(a, b, c, alpha, count, vec);
  }
  return st_of(cudaGetLastError());
}

template <int KIND>
__global__ void k_to_half(const float *x, uint16_t *h, int64_t count) {
  const int64_t nth = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += nth)
    h[i] = f2h<KIND>(x[i]);
}

template <int KIND>
__global__ void k_from_half(const uint16_t *h, float *x, int64_t count) {
  const int64_t nth = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += nth)
    x[i] = h2f<KIND>(h[i]);
}

// ------------------------------------------------------------- error stats

__device__ __forceinline__ void atomic_max_nonneg(double *addr, double v) {
  // non-negative doubles order like their bit patterns
  atomicMax(reinterpret_cast<unsigned long long *>(addr), (unsigned long long)__double_as_longlong(v));
}

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ double warp_max(double v) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

__global__ void __launch_bounds__(256) k_error_stats(const float *__restrict__ x,
                                                     const float *__restrict__ xh, int64_t n,
                                                     double *out) {
  double acc[IVC_STATS_LEN];
  for (int k = 0; k < IVC_STATS_LEN; ++k) acc[k] = 0.0;
  const int64_t nth = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += nth) {
    const double a0 = x[3 * i], a1 = x[3 * i + 1], a2 = x[3 * i + 2];
    if (!isfinite(a0) || !isfinite(a1) || !isfinite(a2)) continue;
    const double na = sqrt(a0 * a0 + a1 * a1 + a2 * a2);
    if (na == 0.0) continue;
    const double b0 = xh[3 * i], b1 = xh[3 * i + 1], b2 = xh[3 * i + 2];
    if (!isfinite(b0) || !isfinite(b1) || !isfinite(b2)) {
      acc[10] += 1.0;
      continue;
    }
    const double d0 = a0 - b0, d1 = a1 - b1, d2 = a2 - b2;
    const double e = sqrt(d0 * d0 + d1 * d1 + d2 * d2);
    const double nb = sqrt(b0 * b0 + b1 * b1 + b2 * b2);
    const double c0 = a1 * b2 - a2 * b1, c1 = a2 * b0 - a0 * b2, c2 = a0 * b1 - a1 * b0;
    const double ang = atan2(sqrt(c0 * c0 + c1 * c1 + c2 * c2), a0 * b0 + a1 * b1 + a2 * b2);
    const double rel = fabs(nb - na) / na;
    acc[0] += 1.0;
    acc[1] += e;
    acc[2] += e * e;
    acc[3] = fmax(acc[3], e);
    acc[4] += e / na;
    acc[5] = fmax(acc[5], e / na);
    acc[6] += ang * ang;
    acc[7] = fmax(acc[7], ang);
    acc[8] += rel * rel;
    acc[9] = fmax(acc[9], rel);
  }
  __shared__ double red[IVC_STATS_LEN][8];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int k = 0; k < IVC_STATS_LEN; ++k) {
    const bool is_max = (k == 3 || k == 5 || k == 7 || k == 9);
    const double v = is_max ? warp_max(acc[k]) : warp_sum(acc[k]);
    if (lane == 0) red[k][wid] = v;
  }
  __syncthreads();
  if (threadIdx.x < IVC_STATS_LEN) {
    const int k = threadIdx.x;
    const bool is_max = (k == 3 || k == 5 || k == 7 || k == 9);
    double v = red[k][0];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) v = is_max ? fmax(v, red[k][w]) : v + red[k][w];
    if (is_max) atomic_max_nonneg(out + k, v);
    else atomicAdd(out + k, v);
  }
}

}  // namespace

extern "C" {

ivc_status ivc_f32_add(ivc_layout layout, const float *a, const float *b, float *c, int64_t ld,
                       int64_t n, ivc_stream_t stream) {
  return f32_op(false, layout, 0.0f, a, b, c, ld, n, stream);
}

ivc_status ivc_f32_axpy(ivc_layout layout, float alpha, const float *x, float *y, int64_t ld,
                        int64_t n, ivc_stream_t stream) {
  return f32_op(true, layout, alpha, x, y, y, ld, n, stream);
}

ivc_status ivc_f32_gather(ivc_layout layout, const float *src, int64_t ld, int64_t nsrc,
                          const int64_t *idx, int64_t n, float *out, ivc_stream_t stream) {
  if (n < 0 || nsrc < 0 || (layout != IVC_AOS && layout != IVC_SOA)) return IVC_ERR_ARG;
  if (layout == IVC_SOA && ld < nsrc) return IVC_ERR_ARG;
  if (n == 0) return IVC_OK;
  if (!idx || !out || (nsrc > 0 && !src)) return IVC_ERR_ARG;
  if ((src && !aligned(src, 4)) || !aligned(idx, 8) || !aligned(out, 4)) return IVC_ERR_ALIGN;
  const int grid = grid_for(n, 256, 8);
  if (layout == IVC_SOA)
    k_f32_gather<true><<<grid, 256, 0, stream>>>(src, ld, nsrc, idx, n, out);
  else
    k_f32_gather<false><<<grid, 256, 0, stream>>>(src, ld, nsrc, idx, n, out);
  return st_of(cudaGetLastError());
}

ivc_status ivc_half_add(ivc_half_kind kind, const uint16_t *a, const uint16_t *b, uint16_t *c,
                        int64_t n, ivc_stream_t stream) {
  return half_op(false, kind, 0.0f, a, b, c, n, stream);
}

ivc_status ivc_half_axpy(ivc_half_kind kind, float alpha, const uint16_t *x, uint16_t *y,
                         int64_t n, ivc_stream_t stream) {
  return half_op(true, kind, alpha, x, y, y, n, stream);
}

ivc_status ivc_half_from_f32(ivc_half_kind kind, const float *xyz, uint16_t *h, int64_t n,
                             ivc_stream_t stream) {
  if (n < 0 || (kind != IVC_F16 && kind != IVC_BF16)) return IVC_ERR_ARG;
  if (n == 0) return IVC_OK;
  if (!xyz || !h) return IVC_ERR_ARG;
  if (!aligned(xyz, 4) || !aligned(h, 2)) return IVC_ERR_ALIGN;
  const int grid = grid_for(3 * n, 256, 8);
  if (kind == IVC_F16) k_to_half<IVC_F16><<<grid, 256, 0, stream>>>(xyz, h, 3 * n);
  else k_to_half<IVC_BF16><<<grid, 256, 0, stream>>>(xyz, h, 3 * n);
  return st_of(cudaGetLastError());
}

ivc_status ivc_half_to_f32(ivc_half_kind kind, const uint16_t *h, float *xyz, int64_t n,
                           ivc_stream_t stream) {
  if (n < 0 || (kind != IVC_F16 && kind != IVC_BF16)) return IVC_ERR_ARG;
  if (n == 0) return IVC_OK;
  if (!xyz || !h) return IVC_ERR_ARG;
  if (!aligned(xyz, 4) || !aligned(h, 2)) return IVC_ERR_ALIGN;
  const int grid = grid_for(3 * n, 256, 8);
  if (kind == IVC_F16) k_from_half<IVC_F16><<<grid, 256, 0, stream>>>(h, xyz, 3 * n);
  else k_from_half<IVC_BF16><<<grid, 256, 0, stream>>>(h, xyz, 3 * n);
  return st_of(cudaGetLastError());
}

ivc_status ivc_error_stats(const float *x, const float *xh, int64_t n, double *out,
                           ivc_stream_t stream) {
  if (n < 0) return IVC_ERR_ARG;
  if (n == 0) return IVC_OK;
  if (!x || !xh || !out) return IVC_ERR_ARG;
  if (!aligned(x, 4) || !aligned(xh, 4) || !aligned(out, 8)) return IVC_ERR_ALIGN;
  const int grid = grid_for(n, 256, 4);
  k_error_stats<<<grid, 256, 0, stream>>>(x, xh, n, out);
  return st_of(cudaGetLastError());
}

}  // extern "C"
