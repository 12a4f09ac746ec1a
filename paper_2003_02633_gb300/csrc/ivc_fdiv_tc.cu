// Divergence of a compressed flux (Algorithm 1, Sec. 4; Table fr_nse step 10)
// on the fifth-generation tensor cores.
//
// The contraction div(k, p, e) = sum_j sum_c D[c ns + j][k] X(j, p, e)_c is,
// for one equation p and a tile of 128 elements, the product
//     Out (128 x ns) = A (128 x 3 ns) B (3 ns x ns),
// A[e][3 j + c] = X(j, p, e)_c (the decoded flux) and B[3 j + c][k] =
// D[c ns + j][k].  One persistent block per SM stages B once and walks its
// tiles in stages of 8 solution points of one equation: 16 decoding warps
// write a stage's A (K-major, no swizzle: 8-row x 16-byte core matrices) into
// one of 4 shared-memory buffers and arrive on its "full" mbarrier; one thread
// of a 17th warp waits for it, issues tcgen05.mma (M = 128, N = ns padded to
// 16, K = 8 per instruction) into the equation's FP32 accumulator in tensor
// memory, and tcgen05.commit releases the buffer through its "empty"
// mbarrier.  After a tile's last stage, four decoding warps read the
// accumulators (tcgen05.ld) and store the divergence, and the next tile's
// first products wait on an mbarrier until they have.
//
// Precision: the operands are FP32 values with 24-bit significands, so each
// is split into a TF32 head (rounded to nearest) and the FP32 remainder, and
// the product takes three TF32 products (head x head, head x tail, tail x
// head): the dropped tail x tail term and the tails' own truncation to TF32
// are below 2^-20 of |D||X| per term, far inside the FP32 summation bound the
// result is held to; the accumulation is FP32.
//
// Every mbarrier wait is bounded (about a second of clock cycles); a wait that
// runs out sets the device status word read by ivc_flux_divergence_check, and
// the block still waits (bounded) for its own tensor-core work and frees its
// tensor memory before it returns.
#include "ivc_decode_poles.cuh"
#include "ivc_internal.h"

namespace ivc {
namespace {

constexpr int kTM = 128;             // elements per tile (the MMA's M)
constexpr int kPC = 8;               // solution points per chunk
constexpr int kKC = 3 * kPC;         // K per chunk (3 components per point)
constexpr int kKStepsC = kKC / 8;    // K = 8 per tf32 MMA
constexpr int kCoreBytes = 128;      // one 8-row x 16-byte core matrix
constexpr int kAStep = (kTM / 8) * 2 * kCoreBytes;       // bytes of A per K step
constexpr int kABuf = kKStepsC * kAStep;                 // one A buffer (head or tail)
constexpr long long kWaitCycles = 2000000000ll;
constexpr uint32_t kSuspendNs = 65536;
constexpr int kMaxNs = 64;
constexpr int kMaxNv = 5;

enum : int { TC_GENERIC = 0, TC_FAST = 1, TC_F32 = 2 };

__device__ int g_fdiv_tc_status;

__host__ __device__ constexpr int pad_to(int v, int m) { return (v + m - 1) / m * m; }

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// Shared-memory matrix descriptor: K-major, no swizzle; lbo = byte step between
// core matrices along K, sbo = byte step between 8-row groups.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)(lbo >> 4) << 16) |
         ((uint64_t)(sbo >> 4) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::tf32: FP32 accumulator, TF32 A and B, both
// K-major, N >> 3 and M >> 4.
__host__ __device__ constexpr uint32_t idesc_tf32(int m, int n) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) |
         ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t *bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void fence_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void bar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}

// Bounded wait for the completion of the phase with the given parity.  Each
// try_wait may suspend the thread for up to kSuspendNs until the phase
// completes, instead of returning at once, so a waiting warp issues few
// instructions.
__device__ __forceinline__ bool bar_wait(uint64_t *bar, uint32_t parity) {
  const uint32_t a = smem_u32(bar);
  const long long t0 = clock64();
  while (true) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.b32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(a), "r"(parity), "r"(kSuspendNs)
        : "memory");
    if (ok) return true;
    if (clock64() - t0 > kWaitCycles) return false;
  }
}

// 32 consecutive accumulator columns of this warp's 32 lanes.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float v[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
      "%11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, "
      "%28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
        "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
        "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
        "=r"(r[31])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// TF32 head (rounded to nearest) and FP32 tail of x.
__device__ __forceinline__ void split_tf32(float x, float &hi, float &lo) {
  uint32_t h;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(h) : "f"(x));
  hi = __uint_as_float(h);
  lo = x - hi;
}

// Byte offset of entry (row, k) of a K-major no-swizzle operand whose K step
// holds `rows` rows: core matrix (row / 8, k % 8 / 4) of K step k / 8.
__device__ __forceinline__ uint32_t kmajor_off(int row, int k, int rows) {
  return (uint32_t)((k >> 3) * (rows / 8) * 2 * kCoreBytes + (row >> 3) * 2 * kCoreBytes +
                    ((k >> 2) & 1) * kCoreBytes + (row & 7) * 16 + (k & 3) * 4);
}

constexpr int kProducers = 512;               // 16 decoding warps, one element pair each
constexpr int kThreadsTC = kProducers + 32;    // + the warp that issues the products
// Stage shape per row type: compressed rows decode one equation per stage
// into one of 4 buffers; FP32 rows, whose stages are only loads, take two
// equations per stage (two buffers), fewer and longer stages being faster there.
template <int MODE>
struct TcShape {
  static constexpr int kVPS = MODE == TC_F32 ? 2 : 1;     // equations per stage
  static constexpr int kStages = MODE == TC_F32 ? 2 : 4;  // A buffers in flight (power of 2)
};

// Shared memory: [B head | B tail | A stages (head, tail) | tables |
//                 barriers full[S], empty[S], acc_full, acc_empty | TMEM address | abort]
struct TcLayout {
  int nsp, np, kt;           // points padded to 8, N (= ns padded to 16), K = 3 nsp
  uint32_t b_bytes;          // one B copy
  uint32_t off_a, off_tab, off_bar, total;
};

template <int MODE>
__host__ __device__ inline TcLayout tc_layout(int ns, int ntab_bytes) {
  constexpr int kVPS = TcShape<MODE>::kVPS, kStages = TcShape<MODE>::kStages;
  TcLayout L;
  L.nsp = pad_to(ns, kPC);
  L.np = pad_to(ns, 16);
  L.kt = 3 * L.nsp;
  L.b_bytes = (uint32_t)(L.kt / 8) * (L.np / 8) * 2 * kCoreBytes;
  L.off_a = 2 * L.b_bytes;
  L.off_tab = L.off_a + kStages * kVPS * 2 * kABuf;
  L.off_bar = L.off_tab + (uint32_t)pad_to(ntab_bytes, 16);
  L.total = L.off_bar + (2 * kStages + 2) * 8 + 16;
  return L;
}

__device__ __forceinline__ void bar_arrive(uint64_t *bar) {
  asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(
                   smem_u32(bar))
               : "memory");
}

// The stage of a block's global stage counter g: its tile (of this block's
// tiles), point chunk ch and first equation p (VPS equations per stage).
template <int VPS>
struct Stage {
  int64_t tile;
  int64_t ti;        // index of the tile among the block's tiles
  int ch, p;
  bool first, last;  // first / last stage of the tile

  __device__ void start(int nchunk, int nv) {
    ti = 0;
    tile = blockIdx.x;
    ch = 0;
    p = 0;
    first = true;
    last = nchunk == 1 && VPS >= nv;
  }
  // the next stage: equation, then point chunk, then the block's next tile
  __device__ void advance(int nchunk, int nv) {
    p += VPS;
    if (p >= nv) {
      p = 0;
      if (++ch == nchunk) {
        ch = 0;
        ++ti;
        tile += gridDim.x;
      }
    }
    first = ch == 0 && p == 0;
    last = ch == nchunk - 1 && p + VPS >= nv;
  }
};

// A producer's pair of stage s: point jj = lane / 8 + 4 (warp / 8), elements
// m = 8 (warp % 8) + lane % 8 and m + 64 of the tile.  Within a warp the
// stores into A fall on 32 distinct banks (8 rows x 4 columns of a core
// matrix) and the loads are runs of 8 consecutive elements.
template <int MODE>
struct PairIn {
  static constexpr int V = TcShape<MODE>::kVPS;
  float a[V][3], b[V][3];
  uint64_t w0[V], w1[V];
};

template <int MODE>
__device__ __forceinline__ void load_pair(PairIn<MODE> &in, const void *src, int64_t ld, int ns,
                                          int nv, int64_t ne,
                                          const Stage<TcShape<MODE>::kVPS> &s, int jj, int m) {
  const int j = s.ch * kPC + jj;
  const int64_t ea = s.tile * kTM + m, eb = ea + kTM / 2;
#pragma unroll
  for (int v = 0; v < PairIn<MODE>::V; ++v) {
    const bool pv = s.p + v < nv;
    const bool va = pv && j < ns && ea < ne, vb = pv && j < ns && eb < ne;
    const int64_t row = ((int64_t)(j < ns ? j : 0) * nv + (pv ? s.p + v : 0)) * ld;
    if (MODE == TC_F32) {
      const float *Fr = static_cast<const float *>(src);
      const int64_t cs = (int64_t)ns * nv * ld;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        in.a[v][c] = va ? __ldg(Fr + row + c * cs + ea) : 0.0f;
        in.b[v][c] = vb ? __ldg(Fr + row + c * cs + eb) : 0.0f;
      }
    } else {
      const uint64_t *W = static_cast<const uint64_t *>(src);
      in.w0[v] = va ? __ldg(W + row + ea) : 0ull;
      in.w1[v] = vb ? __ldg(W + row + eb) : 0ull;
    }
  }
}

template <int MODE, int MAP>
__global__ void __launch_bounds__(kThreadsTC, 1)
    k_flux_div_tc(const __grid_constant__ DevFormat F, const void *__restrict__ src, int64_t ld,
                  int ns, int nv, int64_t ne, const float *__restrict__ D,
                  float *__restrict__ div, int64_t ld_out, uint32_t tmem_cols) {
  extern __shared__ __align__(1024) unsigned char smem[];
  const int ntab = (MODE == TC_F32 || MAP == MAP_TANH) ? 0 : F.nent_t + F.nent_p;
  constexpr int kVPS = TcShape<MODE>::kVPS, kStages = TcShape<MODE>::kStages;
  using StageT = Stage<kVPS>;
  const TcLayout L = tc_layout<MODE>(ns, ntab * (int)sizeof(TabEntry));
  unsigned char *Bh = smem, *Bl = smem + L.b_bytes;
  unsigned char *Abase = smem + L.off_a;
  TabEntry *tabs = reinterpret_cast<TabEntry *>(smem + L.off_tab);
  uint64_t *full = reinterpret_cast<uint64_t *>(smem + L.off_bar);
  uint64_t *empty = full + kStages;
  uint64_t *acc_full = empty + kStages, *acc_empty = acc_full + 1;
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(acc_empty + 1);
  volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t ntiles = (ne + kTM - 1) / kTM;
  const int nchunk = pad_to(ns, kPC) / kPC;
  const int nq = nchunk * ((nv + kVPS - 1) / kVPS);
  const int64_t my_tiles = (int64_t)blockIdx.x < ntiles
                               ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  const int64_t niter = my_tiles * nq;
  const bool producer = threadIdx.x < kProducers;
  const int jj = (lane >> 3) + 4 * (warp >> 3), m = 8 * (warp & 7) + (lane & 7);

  // the first two stages' loads go out before the set-up
  PairIn<MODE> cur, nxt;
  StageT ls;                                    // the stage of the next loads
  ls.start(nchunk, nv);
  if (producer) {
    if (niter > 0) load_pair<MODE>(cur, src, ld, ns, nv, ne, ls, jj, m);
    ls.advance(nchunk, nv);
    if (niter > 1) load_pair<MODE>(nxt, src, ld, ns, nv, ne, ls, jj, m);
    ls.advance(nchunk, nv);
  }
  if (warp == kProducers / 32) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (threadIdx.x == 0) {
    for (int i = 0; i < kStages; ++i) {
      bar_init(full + i, kProducers);
      bar_init(empty + i, 1);
    }
    bar_init(acc_full, 1);
    bar_init(acc_empty, 4 * 32);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (ntab > 0) stage_tables<MAP>(F, tabs);
  const TabEntry *tab_t = tabs;
  const TabEntry *tab_p = tabs + (MAP == MAP_TANH ? 0 : F.nent_t);
  // B = the operator, K index 3 j + c, N index k, head and tail; zero padding
  for (int i = threadIdx.x; i < L.kt * L.np; i += kThreadsTC) {
    const int k = i % L.np, kk = i / L.np;
    const int j = kk / 3, c = kk - 3 * j;
    const float d = (j < ns && k < ns) ? __ldg(D + (int64_t)(c * ns + j) * ns + k) : 0.0f;
    float hi, lo;
    split_tf32(d, hi, lo);
    const uint32_t off = kmajor_off(k, kk, L.np);
    *reinterpret_cast<float *>(Bh + off) = hi;
    *reinterpret_cast<float *>(Bl + off) = lo;
  }
  fence_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (producer) {
    // ------------------------------------------------------------ producers
    // this thread's A offsets (the same in every stage)
    uint32_t offa[3], offb[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      offa[c] = kmajor_off(m, 3 * jj + c, kTM);
      offb[c] = kmajor_off(m + kTM / 2, 3 * jj + c, kTM);
    }
    StageT s;
    s.start(nchunk, nv);
    for (int64_t g = 0; g < niter; ++g, s.advance(nchunk, nv)) {
      const int b = (int)(g & (kStages - 1));
      const uint32_t u = (uint32_t)(g / kStages);
      // loads two stages ahead
      PairIn<MODE> nxt2 = nxt;
      if (g + 2 < niter) load_pair<MODE>(nxt2, src, ld, ns, nv, ne, ls, jj, m);
      ls.advance(nchunk, nv);
      if (u >= 1 && !bar_wait(empty + b, (u - 1) & 1u)) *abort_flag = 1;
      if (*abort_flag) break;
#pragma unroll
      for (int v = 0; v < kVPS; ++v) {
        float xa[3], xb[3];
        if (MODE == TC_F32) {
#pragma unroll
          for (int c = 0; c < 3; ++c) xa[c] = cur.a[v][c], xb[c] = cur.b[v][c];
        } else {
          float2 X, Y, Z;
          if (MODE == TC_FAST) {
            fast::decode2_f32<fast::GeoPrimary>(cur.w0[v], cur.w1[v], F, tab_t, tab_p, X, Y,
                                                Z);
          } else {
            const float3 a0 = decode_word<MAP>(cur.w0[v], F, tab_t, tab_p);
            const float3 a1 = decode_word<MAP>(cur.w1[v], F, tab_t, tab_p);
            X = make_float2(a0.x, a1.x);
            Y = make_float2(a0.y, a1.y);
            Z = make_float2(a0.z, a1.z);
          }
          xa[0] = X.x, xa[1] = Y.x, xa[2] = Z.x;
          xb[0] = X.y, xb[1] = Y.y, xb[2] = Z.y;
        }
        unsigned char *Ah = Abase + (b * kVPS + v) * 2 * kABuf, *Al = Ah + kABuf;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          float hi, lo;
          split_tf32(xa[c], hi, lo);
          *reinterpret_cast<float *>(Ah + offa[c]) = hi;
          *reinterpret_cast<float *>(Al + offa[c]) = lo;
          split_tf32(xb[c], hi, lo);
          *reinterpret_cast<float *>(Ah + offb[c]) = hi;
          *reinterpret_cast<float *>(Al + offb[c]) = lo;
        }
      }
      fence_async_smem();
      bar_arrive(full + b);
      cur = nxt;
      nxt = nxt2;
      if (s.last && warp < 4) {
        // epilogue of the tile: the accumulators, once its products are done
        if (!bar_wait(acc_full, (uint32_t)(s.ti & 1))) *abort_flag = 1;
        if (*abort_flag) break;
        tc_fence_after();
        const int64_t e = s.tile * kTM + warp * 32 + lane;
        for (int p = 0; p < nv; ++p) {
          for (int c0 = 0; c0 < L.np; c0 += 32) {
            float v[32];
            tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(p * L.np + c0), v);
            if (e < ne) {
#pragma unroll
              for (int i = 0; i < 32; ++i) {
                const int k = c0 + i;
                if (k < ns) div[((int64_t)k * nv + p) * ld_out + e] = v[i];
              }
            }
          }
        }
        tc_fence_before();
        bar_arrive(acc_empty);
      }
    }
  } else if (lane == 0) {
    // -------------------------------------------------------- the MMA issuer
    const uint32_t idesc = idesc_tf32(kTM, L.np);
    int64_t issued = -1;                       // last stage with products in flight
    StageT s;
    s.start(nchunk, nv);
    for (int64_t g = 0; g < niter; ++g, s.advance(nchunk, nv)) {
      const int b = (int)(g & (kStages - 1));
      const uint32_t u = (uint32_t)(g / kStages);
      if (!bar_wait(full + b, u & 1u)) *abort_flag = 1;
      // a new tile overwrites the accumulators: the previous tile's epilogue
      // must have read them
      if (s.first && s.ti >= 1 && !*abort_flag && !bar_wait(acc_empty, (uint32_t)((s.ti - 1) & 1)))
        *abort_flag = 1;
      if (*abort_flag) break;
      tc_fence_after();
      for (int v = 0; v < kVPS && s.p + v < nv; ++v) {
        unsigned char *Ah = Abase + (b * kVPS + v) * 2 * kABuf, *Al = Ah + kABuf;
        const uint32_t d = tmem + (uint32_t)((s.p + v) * L.np);
#pragma unroll
        for (int t = 0; t < kKStepsC; ++t) {
          const int st = s.ch * kKStepsC + t;
          const uint64_t ah = smem_desc(smem_u32(Ah + t * kAStep), kCoreBytes, 2 * kCoreBytes);
          const uint64_t al = smem_desc(smem_u32(Al + t * kAStep), kCoreBytes, 2 * kCoreBytes);
          const uint32_t boff = (uint32_t)st * (L.np / 8) * 2 * kCoreBytes;
          const uint64_t bh = smem_desc(smem_u32(Bh + boff), kCoreBytes, 2 * kCoreBytes);
          const uint64_t bl = smem_desc(smem_u32(Bl + boff), kCoreBytes, 2 * kCoreBytes);
          mma_tf32(d, ah, bh, idesc, (s.ch > 0 || t > 0) ? 1u : 0u);
          mma_tf32(d, ah, bl, idesc, 1u);
          mma_tf32(d, al, bh, idesc, 1u);
        }
      }
      mma_commit(empty + b);
      if (s.last) mma_commit(acc_full);
      issued = g;
    }
    // all products done before the memory is freed (the last commit covers
    // every earlier product of this thread)
    if (issued >= 0)
      bar_wait(empty + (int)(issued & (kStages - 1)), (uint32_t)(issued / kStages) & 1u);
  }
  if (*abort_flag && threadIdx.x == 0) atomicExch(&g_fdiv_tc_status, 1);
  tc_fence_before();
  __syncthreads();
  if (warp == kProducers / 32) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(tmem_cols)
                 : "memory");
  }
}

template <int MODE, int MAP>
cudaError_t launch_tc(const DevFormat &F, const void *src, int64_t ld, int ns, int nv, int64_t ne,
                      const float *D, float *div, int64_t ld_out, cudaStream_t st) {
  const int ntab = (MODE == TC_F32 || MAP == MAP_TANH) ? 0 : F.nent_t + F.nent_p;
  const TcLayout L = tc_layout<MODE>(ns, ntab * (int)sizeof(TabEntry));
  // one block per SM (the tensor-memory allocation assumes it): at least
  // 120 KB of shared memory
  const size_t smem = L.total < 120u * 1024u ? 120u * 1024u : L.total;
  // accumulator columns: nv blocks of np, the last read 32 at a time
  uint32_t cols = 32;
  while (cols < (uint32_t)((nv - 1) * L.np + pad_to(L.np, 32))) cols <<= 1;
  const void *k = (const void *)k_flux_div_tc<MODE, MAP>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 1;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
    return e;
  const int64_t ntiles = (ne + kTM - 1) / kTM;
  const int64_t grid = ntiles < sms ? ntiles : sms;       // persistent: one block per SM
  k_flux_div_tc<MODE, MAP><<<(unsigned)grid, kThreadsTC, smem, st>>>(F, src, ld, ns, nv, ne, D,
                                                                      div, ld_out, cols);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_flux_div_tc(int map, bool fast_path, bool f32, const DevFormat &F,
                               const void *src, int64_t ld, int ns, int nv, int64_t ne,
                               const float *D, float *div, int64_t ld_out, cudaStream_t st) {
  if (ns < 1 || ns > kMaxNs || nv < 1 || nv > kMaxNv) return cudaErrorInvalidValue;
  if (f32) return launch_tc<TC_F32, MAP_UNIFORM>(F, src, ld, ns, nv, ne, D, div, ld_out, st);
  if (fast_path) return launch_tc<TC_FAST, MAP_UNIFORM>(F, src, ld, ns, nv, ne, D, div, ld_out, st);
  switch (map) {
    case MAP_UNIFORM:
      return launch_tc<TC_GENERIC, MAP_UNIFORM>(F, src, ld, ns, nv, ne, D, div, ld_out, st);
    case MAP_TANH:
      return launch_tc<TC_GENERIC, MAP_TANH>(F, src, ld, ns, nv, ne, D, div, ld_out, st);
    default:
      return launch_tc<TC_GENERIC, MAP_FRACSPLIT>(F, src, ld, ns, nv, ne, D, div, ld_out, st);
  }
}

cudaError_t flux_div_tc_status(int *status) {
  cudaError_t e = cudaMemcpyFromSymbol(status, g_fdiv_tc_status, sizeof(int));
  if (e != cudaSuccess) return e;
  const int zero = 0;
  return cudaMemcpyToSymbol(g_fdiv_tc_status, &zero, sizeof(int));
}

}  // namespace ivc
