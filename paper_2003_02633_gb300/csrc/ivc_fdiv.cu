// Divergence of a compressed flux: Algorithm 1 (Sec. 4; Table fr_nse, step
// 10).  For each element and solution point k:
//     div(k, p) = sum_j sum_c D[c ns + j][k] X(j, p)_c,   X = decompress(F).
//
// GB300 layout of the work: a block owns a tile of 64 elements and all ns
// output points, and splits its warps by role.  Eight producer warps take the
// words of 8 solution points at a time (8 x nvars rows x 64 elements,
// coalesced along the element index): they copy the next chunk's words into
// shared memory with asynchronous copies (cp.async) while decoding the current
// chunk's words into one of two shared-memory buffers as FP32.  Eight
// consumer warps accumulate, per thread, a 4 (points k) x nvars x 4
// (elements) block of the output with FP32 FMAs from the other buffer and
// from D (staged once per block).  Two mbarriers per buffer ("full": the
// producers' arrivals, "empty": the consumers') hand the buffers back and
// forth, so decoding the next points overlaps the FMAs of the current ones,
// and the 80 accumulators never share a thread with the decoder's registers.
// Every wait is bounded (about a second of clock cycles); a wait that runs
// out marks the launch failed in a device status word and the block leaves.
//
// The contraction has K = 3 ns = 192 terms per output for hex elements of
// degree 3; it runs on the FP32 pipes because its operands carry 24-bit
// significands and the result is held to an FP32 summation bound (a TF32 or
// BF16 tensor-core product would round the decoded flux to 11 or 8 bits).
#include "ivc_decode_poles.cuh"
#include "ivc_internal.h"

namespace ivc {
namespace {

constexpr int kTE = 64;         // elements per tile
constexpr int kJC = 8;          // solution points per chunk
constexpr int kMaxNs = 64;
constexpr int kMaxNv = 5;
constexpr int kProducers = 256; // 8 warps
constexpr int kConsumers = 256; // 8 warps
constexpr int kThreads = kProducers + kConsumers;
constexpr int kXBuf = kJC * kMaxNv * 3 * kTE;   // floats per decoded buffer
constexpr int kWBuf = kJC * kMaxNv * kTE * 3;   // 32-bit units per raw buffer (FP32 rows)
constexpr long long kWaitCycles = 2000000000ll; // default bound of each wait: about a second
// the bound every launch gets (ivc_set_flux_divergence_wait_limit)
long long g_wait_cycles = kWaitCycles;
// the consumers cover 64 points (16 groups of 4) x the tile's elements (groups of 4)
static_assert(kConsumers == 16 * (kTE / 4), "consumer mapping");
static_assert(kProducers % (kTE / 2) == 0, "producer mapping");

enum : int { FD_GENERIC = 0, FD_FAST = 1, FD_F32 = 2 };

__device__ int g_fdiv_status;  // 0 ok, 1 a bounded wait ran out

__host__ __device__ constexpr int pad4(int v) { return (v + 3) & ~3; }

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(
                   smem_addr(bar))
               : "memory");
}

// 4- or 8-byte asynchronous global-to-shared copy; bytes = 0 fills zeros
// without reading the source.
template <int SIZE>
__device__ __forceinline__ void cp_async(void *dst, const void *src, uint32_t bytes) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;" ::"r"(smem_addr(dst)),
               "l"(__cvta_generic_to_global(src)), "n"(SIZE), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;" ::: "memory");
}

__device__ __forceinline__ void cp_async_wait_1() {
  asm volatile("cp.async.wait_group 1;" ::: "memory");
}

__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_all;" ::: "memory");
}

// Waits for the completion of the barrier phase with the given parity;
// false when `limit` cycles (about a second by default) passed first.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, long long limit) {
  const uint32_t a = smem_addr(bar);
  const long long t0 = clock64();
  while (true) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.b32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(a), "r"(parity)
        : "memory");
    if (ok) return true;
    if (clock64() - t0 > limit) return false;
  }
}

// Rows of a chunk handled by one producer thread: the thread owns the element
// pair e2 = pt % (kTE / 2) of the rows r = pt / (kTE / 2) + kRowsPass t
// (t < kRowsPT), row r being
// point jj = r / nvars, equation p = r % nvars of the chunk.  The same thread
// copies and later decodes each of its items, so it waits only for its own
// cp.async groups.
constexpr int kRowsPass = kProducers / (kTE / 2);   // rows the producers cover per pass
constexpr int kRowsPT = (kJC * kMaxNv + kRowsPass - 1) / kRowsPass;

struct ProdRows {
  int e2;
  int r[kRowsPT], jj[kRowsPT];
};

__device__ __forceinline__ ProdRows prod_rows(int pt, int nv) {
  ProdRows m;
  m.e2 = pt & (kTE / 2 - 1);
#pragma unroll
  for (int t = 0; t < kRowsPT; ++t) {
    const int r = pt / (kTE / 2) + kRowsPass * t;
    m.r[t] = r;
    m.jj[t] = r / nv;
  }
  return m;
}

// Copies the raw data of one chunk (words, or FP32 components) into a raw
// buffer: item q = r * 32 + e2 (two adjacent elements of row r) at q * 2
// words, or at q * 6 floats (component-major pairs).
template <int MODE>
__device__ __forceinline__ void copy_chunk(uint32_t *Wb, const void *src, int64_t ld, int ns,
                                           int nv, int64_t ne, int64_t e0, int j0, int jn,
                                           const ProdRows &m) {
  const int64_t e = e0 + 2 * m.e2;
  const bool in0 = e < ne, in1 = e + 1 < ne;
#pragma unroll
  for (int t = 0; t < kRowsPT; ++t) {
    if (m.jj[t] >= jn) continue;
    const int q = m.r[t] * (kTE / 2) + m.e2;
    if (MODE == FD_F32) {
      const float *Fr = static_cast<const float *>(src);
      const int jp = (j0 + m.jj[t]) * nv + (m.r[t] - m.jj[t] * nv);   // row within a component
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const int64_t base = ((int64_t)c * ns * nv + jp) * ld + e;
        cp_async<4>(Wb + q * 6 + c * 2, in0 ? (const void *)(Fr + base) : src, in0 ? 4u : 0u);
        cp_async<4>(Wb + q * 6 + c * 2 + 1, in1 ? (const void *)(Fr + base + 1) : src,
                    in1 ? 4u : 0u);
      }
    } else {
      const uint64_t *W = static_cast<const uint64_t *>(src);
      const int64_t base = ((int64_t)j0 * nv + m.r[t]) * ld + e;
      cp_async<8>(Wb + q * 4, in0 ? (const void *)(W + base) : src, in0 ? 8u : 0u);
      cp_async<8>(Wb + q * 4 + 2, in1 ? (const void *)(W + base + 1) : src, in1 ? 8u : 0u);
    }
  }
  cp_async_commit();
}

// Shared memory: [tables][D: 3 ns x pad4(ns)][X: 2 x kXBuf][raw: 2 x kWBuf]
//                [full[2], empty[2]][abort]
template <int MODE, int MAP>
__global__ void __launch_bounds__(kThreads, 1)
    k_flux_div(const __grid_constant__ DevFormat F, const void *__restrict__ src, int64_t ld,
               int ns, int nv, int64_t ne, const float *__restrict__ D, float *__restrict__ div,
               int64_t ld_out, long long wait_limit) {
  extern __shared__ __align__(16) unsigned char fd_smem[];
  TabEntry *tabs = reinterpret_cast<TabEntry *>(fd_smem);
  const int ntab = (MODE == FD_F32 || MAP == MAP_TANH) ? 0 : F.nent_t + F.nent_p;
  const int nsp = pad4(ns);
  float *Ds = reinterpret_cast<float *>(fd_smem + (size_t)ntab * sizeof(TabEntry));
  float *Xs = Ds + 3 * ns * nsp;
  uint32_t *Ws = reinterpret_cast<uint32_t *>(Xs + 2 * kXBuf);
  uint64_t *bars = reinterpret_cast<uint64_t *>(Ws + 2 * kWBuf);  // full[0..1], empty[0..1]
  volatile int *abort_flag = reinterpret_cast<volatile int *>(bars + 4);

  if (ntab > 0) stage_tables<MAP>(F, tabs);
  const TabEntry *tab_t = tabs;
  const TabEntry *tab_p = tabs + (MAP == MAP_TANH ? 0 : F.nent_t);
  for (int i = threadIdx.x; i < 3 * ns * nsp; i += kThreads) {
    const int r = i / nsp, k = i - r * nsp;
    Ds[i] = k < ns ? D[(int64_t)r * ns + k] : 0.0f;
  }
  if (threadIdx.x == 0) {
    mbar_init(bars + 0, kProducers);
    mbar_init(bars + 1, kProducers);
    mbar_init(bars + 2, kConsumers);
    mbar_init(bars + 3, kConsumers);
    *abort_flag = 0;
  }
  __syncthreads();

  const int64_t ntiles = (ne + kTE - 1) / kTE;
  const int nchunk = (ns + kJC - 1) / kJC;

  if (threadIdx.x < kProducers) {
    // ------------------------------------------------------------ producers
    const ProdRows m = prod_rows(threadIdx.x, nv);
    uint32_t g = 0;
    int64_t tile = blockIdx.x;
    int ch = 0;
    if (tile < ntiles)
      copy_chunk<MODE>(Ws, src, ld, ns, nv, ne, tile * kTE, 0, min(kJC, ns), m);
    while (tile < ntiles) {
      // start the copies of the next chunk, then wait for this chunk's
      int64_t ntile = tile;
      int nch = ch + 1;
      if (nch == nchunk) {
        nch = 0;
        ntile += gridDim.x;
      }
      if (ntile < ntiles)
        copy_chunk<MODE>(Ws + ((g + 1) & 1) * kWBuf, src, ld, ns, nv, ne, ntile * kTE,
                         nch * kJC, min(kJC, ns - nch * kJC), m);
      else
        cp_async_commit();  // an empty group keeps "all but the newest" meaning this chunk
      cp_async_wait_1();
      const int b = g & 1;
      const uint32_t u = g >> 1;
      if (u >= 1 && !mbar_wait(bars + 2 + b, (u - 1) & 1u, wait_limit)) {
        *abort_flag = 1;
        atomicExch(&g_fdiv_status, 1);
        cp_async_wait_all();  // no copy of this thread outlives it
        return;
      }
      if (*abort_flag) {
        cp_async_wait_all();
        return;
      }
      const int jn = min(kJC, ns - ch * kJC);
      float *X = Xs + b * kXBuf;
      const uint32_t *Wb = Ws + b * kWBuf;
      // rows r0 + 8 t in increasing order (so are their points jj): a rolled
      // loop keeps one copy of the decoder in the instruction stream
      int rr = m.r[0], jr = m.jj[0], pr = m.r[0] - m.jj[0] * nv;
#pragma unroll 1
      for (int t = 0; t < kRowsPT && jr < jn; ++t) {
        const int q = rr * (kTE / 2) + m.e2;
        float2 vx, vy, vz;
        if (MODE == FD_F32) {
          vx = *reinterpret_cast<const float2 *>(Wb + q * 6);
          vy = *reinterpret_cast<const float2 *>(Wb + q * 6 + 2);
          vz = *reinterpret_cast<const float2 *>(Wb + q * 6 + 4);
        } else {
          const ulonglong2 w = *reinterpret_cast<const ulonglong2 *>(Wb + q * 4);
          if (MODE == FD_FAST) {
            fast::decode2_poles<fast::GeoPrimary>(w.x, w.y, F, tab_t, tab_p, vx, vy, vz);
          } else {
            const float3 a = decode_word<MAP>(w.x, F, tab_t, tab_p);
            const float3 c3 = decode_word<MAP>(w.y, F, tab_t, tab_p);
            vx = make_float2(a.x, c3.x);
            vy = make_float2(a.y, c3.y);
            vz = make_float2(a.z, c3.z);
          }
        }
        float *xr = X + ((jr * kMaxNv + pr) * 3) * kTE + 2 * m.e2;
        *reinterpret_cast<float2 *>(xr) = vx;
        *reinterpret_cast<float2 *>(xr + kTE) = vy;
        *reinterpret_cast<float2 *>(xr + 2 * kTE) = vz;
        rr += kRowsPass;
        pr += kRowsPass;
        while (pr >= nv) {
          pr -= nv;
          ++jr;
        }
      }
      mbar_arrive(bars + b);
      tile = ntile;
      ch = nch;
      ++g;
    }
    return;
  }

  // -------------------------------------------------------------- consumers
  const int ct = threadIdx.x - kProducers;
  const int eg = ct % (kTE / 4);   // elements 4 eg .. 4 eg + 3 of the tile
  const int kg = ct / (kTE / 4);   // points 4 kg .. 4 kg + 3
  const bool kact = 4 * kg < nsp;
  uint32_t g = 0;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t e0 = tile * kTE;
    // accumulators in element pairs: packed f32x2 FMAs (same rounding as fmaf)
    float2 acc[4][kMaxNv][2];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int p = 0; p < kMaxNv; ++p) acc[a][p][0] = acc[a][p][1] = make_float2(0.0f, 0.0f);
    for (int ch = 0; ch < nchunk; ++ch, ++g) {
      const int b = g & 1;
      const uint32_t u = g >> 1;
      if (!mbar_wait(bars + b, u & 1u, wait_limit)) {
        *abort_flag = 1;
        atomicExch(&g_fdiv_status, 1);
        return;
      }
      if (*abort_flag) return;
      const int j0 = ch * kJC;
      const int jn = min(kJC, ns - j0);
      const float *X = Xs + b * kXBuf;
      if (kact) {
#pragma unroll
        for (int jj = 0; jj < kJC; ++jj) {
          if (jj < jn) {
#pragma unroll
            for (int c = 0; c < 3; ++c) {
              const float4 d =
                  *reinterpret_cast<const float4 *>(Ds + (c * ns + j0 + jj) * nsp + 4 * kg);
              const float2 dk[4] = {fast::bc(d.x), fast::bc(d.y), fast::bc(d.z), fast::bc(d.w)};
#pragma unroll
              for (int p = 0; p < kMaxNv; ++p) {
                if (p < nv) {
                  const float4 x = *reinterpret_cast<const float4 *>(
                      X + ((jj * kMaxNv + p) * 3 + c) * kTE + 4 * eg);
                  const float2 x01 = make_float2(x.x, x.y), x23 = make_float2(x.z, x.w);
#pragma unroll
                  for (int a = 0; a < 4; ++a) {
                    acc[a][p][0] = fast::fma2(dk[a], x01, acc[a][p][0]);
                    acc[a][p][1] = fast::fma2(dk[a], x23, acc[a][p][1]);
                  }
                }
              }
            }
          }
        }
      }
      mbar_arrive(bars + 2 + b);
    }
    // epilogue: points 4 kg + a < ns, elements e0 + 4 eg + bb < ne
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
          const float v[4] = {acc[a][p][0].x, acc[a][p][0].y, acc[a][p][1].x, acc[a][p][1].y};
          if (e + 3 < ne && (reinterpret_cast<uintptr_t>(o) & 15u) == 0) {
            __stcs(reinterpret_cast<float4 *>(o), make_float4(v[0], v[1], v[2], v[3]));
          } else {
#pragma unroll
            for (int bb = 0; bb < 4; ++bb)
              if (e + bb < ne) o[bb] = v[bb];
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
                      (size_t)2 * kXBuf * sizeof(float) + (size_t)2 * kWBuf * sizeof(uint32_t) +
                      4 * sizeof(uint64_t) + 16;
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
                                                            ld_out, g_wait_cycles);
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

void set_flux_div_wait_limit(long long cycles) {
  g_wait_cycles = cycles > 0 ? cycles : kWaitCycles;
}

cudaError_t flux_div_status(int *status) {
  cudaError_t e = cudaMemcpyFromSymbol(status, g_fdiv_status, sizeof(int));
  if (e != cudaSuccess) return e;
  const int zero = 0;
  return cudaMemcpyToSymbol(g_fdiv_status, &zero, sizeof(int));
}

}  // namespace ivc
