// Compressed-vector kernels: compress, decompress, and the fused
// decompress -> FP32 op -> recompress kernels (Sec. 5: C = A + B), single-field
// and batched (persistent, work-list driven).
//
// Memory access: words move as 16-byte pairs (ulonglong2) with streaming
// cache hints when the pointers are 16-byte aligned; the trigonometric head
// tables of the uniform grids are staged once per block into shared memory.
// Grids are persistent-style grid-stride loops sized from the SM count.
#include <type_traits>

#include "ivc_internal.h"

namespace ivc {

#define IVC_TABLES(F, MAP)                                        \
  extern __shared__ TabEntry ivc_smem_tab[];                      \
  stage_tables<MAP>(F, ivc_smem_tab);                             \
  const TabEntry *tab_t = ivc_smem_tab;                           \
  const TabEntry *tab_p = ivc_smem_tab + (MAP == MAP_TANH ? 0 : F.nent_t)

// Tables of the fast kernels of layout G (the tanh map: the encoder's node
// tables) and their queues.
#define IVC_FAST_TABLES(F, G)                                     \
  extern __shared__ TabEntry ivc_smem_tab[];                      \
  fast::stage_fast_tables<G>(F, ivc_smem_tab);                    \
  const TabEntry *tab_t = ivc_smem_tab;                           \
  const TabEntry *tab_p = ivc_smem_tab + fast::fast_ntab_t<G>(F)
#define IVC_FAST_QUEUE(F, G) ((void *)(ivc_smem_tab + fast::fast_ntab<G>(F)))

// Per-thread range-event counters (overflow, underflow, NaN).
using Events = fast::Events;

// Sums the counters over the warp and adds them to the device counts.
__device__ __forceinline__ void flush_counts(const Events &ev, ivc_counts *counts) {
  if (counts == nullptr) return;
  const unsigned m = __activemask();
  const int lead = __ffs(m) - 1;
  const unsigned o = __reduce_add_sync(m, ev.o);
  const unsigned u = __reduce_add_sync(m, ev.u);
  const unsigned q = __reduce_add_sync(m, ev.q);
  if ((int)(threadIdx.x & 31) == lead) {
    if (o) atomicAdd(&counts->n_overflow, (unsigned long long)o);
    if (u) atomicAdd(&counts->n_underflow, (unsigned long long)u);
    if (q) atomicAdd(&counts->n_nonfinite, (unsigned long long)q);
  }
}

// ------------------------------------------------------------------ compress

// EXACT: every rounding decision through the exact integer helpers.
template <int MAP, bool EXACT = false>
__global__ void __launch_bounds__(256) k_compress(const __grid_constant__ DevFormat F,
                                                  const float *__restrict__ xyz, int layout,
                                                  int64_t ld, int64_t n, uint64_t *w,
                                                  ivc_counts *counts) {
  IVC_TABLES(F, MAP);
  Events ev;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    uint32_t flags = 0;
    float x, y, z;
    if (layout == IVC_AOS) {
      x = __ldcs(xyz + 3 * i);
      y = __ldcs(xyz + 3 * i + 1);
      z = __ldcs(xyz + 3 * i + 2);
    } else {
      x = __ldcs(xyz + i);
      y = __ldcs(xyz + ld + i);
      z = __ldcs(xyz + 2 * ld + i);
    }
    __stcs(reinterpret_cast<unsigned long long *>(w) + i,
           (unsigned long long)encode_vec<MAP, EXACT>(x, y, z, F, tab_t, tab_p, flags));
    ev.add(flags);
  }
  flush_counts(ev, counts);
}

// ---------------------------------------------------------------- decompress

template <int MAP, bool EXACT = false>
__global__ void __launch_bounds__(256) k_decompress(const __grid_constant__ DevFormat F,
                                                    const uint64_t *__restrict__ w, int64_t n,
                                                    float *xyz, int layout, int64_t ld) {
  IVC_TABLES(F, MAP);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const uint64_t word = __ldcs(reinterpret_cast<const unsigned long long *>(w) + i);
    const float3 v = decode_word<MAP, EXACT>(word, F, tab_t, tab_p);
    if (layout == IVC_AOS) {
      __stcs(xyz + 3 * i, v.x);
      __stcs(xyz + 3 * i + 1, v.y);
      __stcs(xyz + 3 * i + 2, v.z);
    } else {
      __stcs(xyz + i, v.x);
      __stcs(xyz + ld + i, v.y);
      __stcs(xyz + 2 * ld + i, v.z);
    }
  }
}

// ------------------------------------------------------------- fused kernels

struct OpAdd {
  __device__ __forceinline__ float3 operator()(float3 a, float3 b) const {
    return make_float3(a.x + b.x, a.y + b.y, a.z + b.z);
  }
};

struct OpAxpy {  // fmaf(alpha, x, y)
  float alpha;
  __device__ __forceinline__ float3 operator()(float3 x, float3 y) const {
    return make_float3(fmaf(alpha, x.x, y.x), fmaf(alpha, x.y, y.y), fmaf(alpha, x.z, y.z));
  }
};

template <int MAP, class Op>
__device__ __forceinline__ uint64_t fused1(uint64_t wa, uint64_t wb, const Op &op,
                                           const DevFormat &F, const TabEntry *tab_t,
                                           const TabEntry *tab_p, uint32_t &flags) {
  const float3 u = decode_word<MAP>(wa, F, tab_t, tab_p);
  const float3 v = decode_word<MAP>(wb, F, tab_t, tab_p);
  const float3 s = op(u, v);
  return encode_vec<MAP>(s.x, s.y, s.z, F, tab_t, tab_p, flags);
}

// out[i] = encode(op(decode(a[i]), decode(b[i]))) over [0, n) with the
// calling block set (grid-stride over `nthreads` threads starting at `tid`).
template <int MAP, class Op>
__device__ __forceinline__ void fused_range(const uint64_t *a, const uint64_t *b, uint64_t *out,
                                            int64_t n, bool vec2, int64_t tid, int64_t nthreads,
                                            const Op &op, const DevFormat &F,
                                            const TabEntry *tab_t, const TabEntry *tab_p,
                                            uint32_t &flags) {
  if (vec2) {
    const int64_t n2 = n >> 1;
    const ulonglong2 *a2 = reinterpret_cast<const ulonglong2 *>(a);
    const ulonglong2 *b2 = reinterpret_cast<const ulonglong2 *>(b);
    ulonglong2 *o2 = reinterpret_cast<ulonglong2 *>(out);
    for (int64_t i = tid; i < n2; i += nthreads) {
      const ulonglong2 wa = __ldcs(a2 + i);
      const ulonglong2 wb = __ldcs(b2 + i);
      ulonglong2 r;
      r.x = fused1<MAP>(wa.x, wb.x, op, F, tab_t, tab_p, flags);
      r.y = fused1<MAP>(wa.y, wb.y, op, F, tab_t, tab_p, flags);
      __stcs(o2 + i, r);
    }
    if ((n & 1) && tid == 0) {
      const int64_t i = n - 1;
      out[i] = fused1<MAP>(a[i], b[i], op, F, tab_t, tab_p, flags);
    }
  } else {
    for (int64_t i = tid; i < n; i += nthreads) {
      const uint64_t wa = __ldcs(reinterpret_cast<const unsigned long long *>(a) + i);
      const uint64_t wb = __ldcs(reinterpret_cast<const unsigned long long *>(b) + i);
      __stcs(reinterpret_cast<unsigned long long *>(out) + i,
             (unsigned long long)fused1<MAP>(wa, wb, op, F, tab_t, tab_p, flags));
    }
  }
}

template <int MAP>
__global__ void __launch_bounds__(256) k_add(const __grid_constant__ DevFormat F,
                                             const uint64_t *a, const uint64_t *b, uint64_t *c,
                                             int64_t n, int vec2) {
  IVC_TABLES(F, MAP);
  uint32_t flags = 0;
  fused_range<MAP>(a, b, c, n, vec2 != 0, (int64_t)blockIdx.x * blockDim.x + threadIdx.x,
                   (int64_t)gridDim.x * blockDim.x, OpAdd{}, F, tab_t, tab_p, flags);
}

template <int MAP>
__global__ void __launch_bounds__(256) k_axpy(const __grid_constant__ DevFormat F, float alpha,
                                              const uint64_t *x, uint64_t *y, int64_t n,
                                              int vec2) {
  IVC_TABLES(F, MAP);
  uint32_t flags = 0;
  fused_range<MAP>(x, y, y, n, vec2 != 0, (int64_t)blockIdx.x * blockDim.x + threadIdx.x,
                   (int64_t)gridDim.x * blockDim.x, OpAxpy{alpha}, F, tab_t, tab_p, flags);
}

// v_out = encode(fmaf(dt, decode(f), decode(v))); m_out = encode(rho * v_new).
template <int MAP>
__global__ void __launch_bounds__(256) k_update(const __grid_constant__ DevFormat F, float dt,
                                                const uint64_t *v, const uint64_t *f,
                                                const float *__restrict__ rho, uint64_t *v_out,
                                                uint64_t *m_out, int64_t n) {
  IVC_TABLES(F, MAP);
  uint32_t flags = 0;
  const bool want_m = (rho != nullptr) && (m_out != nullptr);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const float3 vv = decode_word<MAP>(__ldcs(reinterpret_cast<const unsigned long long *>(v) + i),
                                       F, tab_t, tab_p);
    const float3 ff = decode_word<MAP>(__ldcs(reinterpret_cast<const unsigned long long *>(f) + i),
                                       F, tab_t, tab_p);
    const float3 s = make_float3(fmaf(dt, ff.x, vv.x), fmaf(dt, ff.y, vv.y), fmaf(dt, ff.z, vv.z));
    __stcs(reinterpret_cast<unsigned long long *>(v_out) + i,
           (unsigned long long)encode_vec<MAP>(s.x, s.y, s.z, F, tab_t, tab_p, flags));
    if (want_m) {
      const float q = __ldcs(rho + i);
      __stcs(reinterpret_cast<unsigned long long *>(m_out) + i,
             (unsigned long long)encode_vec<MAP>(q * s.x, q * s.y, q * s.z, F, tab_t, tab_p,
                                                 flags));
    }
  }
}


// ------------------------------------------------------------- fast path
// Primary layout, two vectors per thread, packed FP32x2 arithmetic.  The loop
// trip count is uniform per warp (the encode's exact-test loop votes across
// the warp); lanes past the end work on zero words and store nothing.

// out[i] = encode(op(decode(a[i]), decode(b[i]))) for i in [0, n) by the
// calling threads: warp `warp` of `nwarps` takes word pairs warp*32 + lane,
// (warp + nwarps)*32 + lane, ...; the trip count is uniform per warp.  The odd
// tail element goes to the thread with warp == 0 and lane == 0.  PT: the
// format carries the per-code phi^ table (F.phi_tab).  STG (tanh map): the
// two per-code table entries of every decoded word are copied into shared
// memory by cp.async one iteration ahead (`stage`: two buffers of 8 16-byte
// slots per thread), so that the decode does not wait on its L2 gathers.
template <int OP, class G, bool PT = true, bool STG = false>
__device__ __forceinline__ void fused_fast_range(const uint64_t *a, const uint64_t *b, uint64_t *c,
                                                 int64_t n, int64_t warp, int64_t nwarps, int lane,
                                                 float alpha, const DevFormat &F,
                                                 const TabEntry *tab_t, const TabEntry *tab_p,
                                                 void *qbase, void *stage = nullptr) {
  fast::WarpQueue wq = fast::warp_queue(qbase);
  const int64_t n2 = n >> 1;
  const ulonglong2 *a2 = reinterpret_cast<const ulonglong2 *>(a);
  const ulonglong2 *b2 = reinterpret_cast<const ulonglong2 *>(b);
  ulonglong2 *c2 = reinterpret_cast<ulonglong2 *>(c);
  if constexpr (STG) {
    // words two iterations ahead; slots of a's pair 0-3, b's pair 4-7
    float4 *sbuf = reinterpret_cast<float4 *>(stage);
    const int ss = blockDim.x, t = threadIdx.x;
    const int64_t st = nwarps * 32;
    ulonglong2 ca = make_ulonglong2(0ull, 0ull), cb = ca, na = ca, nb = ca;
    if (warp * 32 + lane < n2) {
      ca = __ldcs(a2 + warp * 32 + lane);
      cb = __ldcs(b2 + warp * 32 + lane);
    }
    if (warp * 32 + lane + st < n2) {
      na = __ldcs(a2 + warp * 32 + lane + st);
      nb = __ldcs(b2 + warp * 32 + lane + st);
    }
    fast::stage_entries<G>(ca.x, ca.y, F, sbuf + t, ss);
    fast::stage_entries<G>(cb.x, cb.y, F, sbuf + 4 * ss + t, ss);
    asm volatile("cp.async.commit_group;" ::: "memory");
    int buf = 0;
    for (int64_t base = warp * 32; base < n2; base += st) {
      const int64_t i = base + lane;
      const bool act = i < n2;
      const ulonglong2 wa = ca, wb = cb;
      ca = na;
      cb = nb;
      if (i + 2 * st < n2) {
        na = __ldcs(a2 + i + 2 * st);
        nb = __ldcs(b2 + i + 2 * st);
      }
      // the next iteration's entries into the other buffer (its previous
      // contents were read by this thread's last iteration), then wait for
      // this iteration's
      float4 *nxt = sbuf + (buf ^ 1) * 8 * ss + t;
      fast::stage_entries<G>(ca.x, ca.y, F, nxt, ss);
      fast::stage_entries<G>(cb.x, cb.y, F, nxt + 4 * ss, ss);
      asm volatile("cp.async.commit_group;" ::: "memory");
      asm volatile("cp.async.wait_group 1;" ::: "memory");
      const fast::Staged sa{sbuf + buf * 8 * ss + t, ss};
      const fast::Staged sb{sbuf + buf * 8 * ss + 4 * ss + t, ss};
      buf ^= 1;
      float2 ux, uy, uz, vx, vy, vz;
      fast::decode2_full<G, PT>(wa.x, wa.y, F, tab_t, tab_p, ux, uy, uz, &sa);
      fast::decode2_full<G, PT>(wb.x, wb.y, F, tab_t, tab_p, vx, vy, vz, &sb);
      float2 sx, sy, sz;
      if (OP == IVC_OP_ADD) {
        sx = fast::add2(ux, vx); sy = fast::add2(uy, vy); sz = fast::add2(uz, vz);
      } else {
        sx = fast::fma2(fast::bc(alpha), ux, vx);
        sy = fast::fma2(fast::bc(alpha), uy, vy);
        sz = fast::fma2(fast::bc(alpha), uz, vz);
      }
      const fast::Enc2 e = fast::encode2<G>(sx, sy, sz, F, tab_t, tab_p);
      if (act) __stcs(c2 + i, make_ulonglong2(e.w0, e.w1));
      fast::push2<G>(wq, act, e, sx, sy, sz, c + 2 * i, F, tab_t, tab_p);
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
  } else {
  // the next iteration's words are loaded before this iteration's arithmetic
  ulonglong2 na = make_ulonglong2(0ull, 0ull), nb = na;
  if (warp * 32 + lane < n2) {
    na = __ldcs(a2 + warp * 32 + lane);
    nb = __ldcs(b2 + warp * 32 + lane);
  }
  for (int64_t base = warp * 32; base < n2; base += nwarps * 32) {
    const int64_t i = base + lane;
    const bool act = i < n2;
    const ulonglong2 wa = na, wb = nb;
    if (i + nwarps * 32 < n2) {
      na = __ldcs(a2 + i + nwarps * 32);
      nb = __ldcs(b2 + i + nwarps * 32);
    }
    float2 ux, uy, uz, vx, vy, vz;
    fast::decode2_full<G, PT>(wa.x, wa.y, F, tab_t, tab_p, ux, uy, uz);
    fast::decode2_full<G, PT>(wb.x, wb.y, F, tab_t, tab_p, vx, vy, vz);
    float2 sx, sy, sz;
    if (OP == IVC_OP_ADD) {
      sx = fast::add2(ux, vx); sy = fast::add2(uy, vy); sz = fast::add2(uz, vz);
    } else {
      sx = fast::fma2(fast::bc(alpha), ux, vx);
      sy = fast::fma2(fast::bc(alpha), uy, vy);
      sz = fast::fma2(fast::bc(alpha), uz, vz);
    }
    const fast::Enc2 e = fast::encode2<G>(sx, sy, sz, F, tab_t, tab_p);
    if (act) __stcs(c2 + i, make_ulonglong2(e.w0, e.w1));
    fast::push2<G>(wq, act, e, sx, sy, sz, c + 2 * i, F, tab_t, tab_p);
  }
  }
  fast::drain<G>(wq, F, tab_t, tab_p);
  if ((n & 1) && warp == 0 && lane == 0) {
    uint32_t flags = 0;
    const int64_t i = n - 1;
    if (OP == IVC_OP_ADD)
      c[i] = fused1<G::MAP>(a[i], b[i], OpAdd{}, F, tab_t, tab_p, flags);
    else
      c[i] = fused1<G::MAP>(a[i], b[i], OpAxpy{alpha}, F, tab_t, tab_p, flags);
  }
}

// Two blocks of 256 per SM: the register budget that leaves (up to 128 per
// thread; 108 used) keeps the codec spill-free and ran faster than three blocks
// at 80 registers (measured).
template <int OP, class G, bool PT>
__global__ void __launch_bounds__(256, 2) k_fused_fast(const __grid_constant__ DevFormat F,
                                                    const uint64_t *a, const uint64_t *b,
                                                    uint64_t *c, int64_t n, float alpha) {
  IVC_FAST_TABLES(F, G);
  constexpr bool kStg = G::MAP == MAP_TANH;
  fused_fast_range<OP, G, PT, kStg>(
      a, b, c, n, ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5,
      ((int64_t)gridDim.x * blockDim.x) >> 5, threadIdx.x & 31, alpha, F, tab_t, tab_p,
      IVC_FAST_QUEUE(F, G),
      (char *)IVC_FAST_QUEUE(F, G) + (blockDim.x >> 5) * fast::kQueueCap * sizeof(fast::PendItem));
}

// Compress n AoS vectors (primary layout), two per thread; counts as in
// k_compress.  Requires a 8-byte aligned xyz and a 16-byte aligned w.
template <class G>
__global__ void __launch_bounds__(256, 3) k_compress_fast(const __grid_constant__ DevFormat F,
                                                       const float *__restrict__ xyz, int64_t n,
                                                       uint64_t *w, ivc_counts *counts) {
  IVC_FAST_TABLES(F, G);
  const int64_t n2 = n >> 1;
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const float2 *v2 = reinterpret_cast<const float2 *>(xyz);
  ulonglong2 *w2 = reinterpret_cast<ulonglong2 *>(w);
  fast::WarpQueue wq = fast::warp_queue(IVC_FAST_QUEUE(F, G));
  Events ev;
  // floats 6i .. 6i+5: x0 y0 z0 x1 y1 z1; the next iteration's are loaded
  // before this iteration's arithmetic
  float2 q0 = make_float2(0.0f, 0.0f), q1 = q0, q2 = q0;
  if (warp * 32 + lane < n2) {
    q0 = __ldcs(v2 + 3 * (warp * 32 + lane));
    q1 = __ldcs(v2 + 3 * (warp * 32 + lane) + 1);
    q2 = __ldcs(v2 + 3 * (warp * 32 + lane) + 2);
  }
  for (int64_t base = warp * 32; base < n2; base += nwarps * 32) {
    const int64_t i = base + lane;
    const bool act = i < n2;
    const float2 p0 = q0, p1 = q1, p2 = q2;
    if (i + nwarps * 32 < n2) {
      q0 = __ldcs(v2 + 3 * (i + nwarps * 32));
      q1 = __ldcs(v2 + 3 * (i + nwarps * 32) + 1);
      q2 = __ldcs(v2 + 3 * (i + nwarps * 32) + 2);
    }
    const float2 vx = make_float2(p0.x, p1.y), vy = make_float2(p0.y, p2.x),
                 vz = make_float2(p1.x, p2.y);
    const fast::Enc2 e = fast::encode2<G>(vx, vy, vz, F, tab_t, tab_p);
    if (act) __stcs(w2 + i, make_ulonglong2(e.w0, e.w1));
    // vectors outside the fast window are encoded (and counted) by the queue
    fast::push2<G>(wq, act, e, vx, vy, vz, w + 2 * i, F, tab_t, tab_p, &ev);
  }
  fast::drain<G>(wq, F, tab_t, tab_p, &ev);
  if ((n & 1) && warp == 0 && lane == 0) {
    const int64_t i = n - 1;
    uint32_t f = 0;
    w[i] = encode_vec<G::MAP>(xyz[3 * i], xyz[3 * i + 1], xyz[3 * i + 2], F, tab_t, tab_p, f);
    ev.add(f);
  }
  flush_counts(ev, counts);
}

// Decompress n words (primary layout) to AoS FP32, two per thread.  Requires
// a 16-byte aligned w and an 8-byte aligned xyz.  With the per-code phi^
// table, each word's phi^ entry is copied into shared memory by cp.async one
// iteration ahead (a decode alone has too little work to hide a direct L2
// gather); otherwise phi^ comes from the shared head table.
template <class G>
__global__ void __launch_bounds__(256, 2) k_decompress_fast(const __grid_constant__ DevFormat F,
                                                         const uint64_t *__restrict__ w,
                                                         int64_t n, float *xyz) {
  IVC_FAST_TABLES(F, G);
  const int64_t n2 = n >> 1;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const ulonglong2 *w2 = reinterpret_cast<const ulonglong2 *>(w);
  float2 *v2 = reinterpret_cast<float2 *>(xyz);
  const int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (G::MAP != MAP_TANH && F.phi_tab) {
    // per-code phi^ entries by cp.async one iteration ahead (two buffers of
    // 4 slots per thread, slots 2 and 3 used), words two iterations ahead
    extern __shared__ TabEntry ivc_smem_tab[];
    float4 *sbuf = reinterpret_cast<float4 *>(ivc_smem_tab + fast::fast_ntab<G>(F));
    const int ss = blockDim.x, t = threadIdx.x;
    ulonglong2 cw = i0 < n2 ? __ldcs(w2 + i0) : make_ulonglong2(0ull, 0ull);
    ulonglong2 nw = i0 + stride < n2 ? __ldcs(w2 + i0 + stride) : make_ulonglong2(0ull, 0ull);
    fast::stage_phi<G>(cw.x, cw.y, F, sbuf + t, ss);
    asm volatile("cp.async.commit_group;" ::: "memory");
    int buf = 0;
    for (int64_t i = i0; i < n2; i += stride) {
      const ulonglong2 ww = cw;
      cw = nw;
      if (i + 2 * stride < n2) nw = __ldcs(w2 + i + 2 * stride);
      fast::stage_phi<G>(cw.x, cw.y, F, sbuf + (buf ^ 1) * 4 * ss + t, ss);
      asm volatile("cp.async.commit_group;" ::: "memory");
      asm volatile("cp.async.wait_group 1;" ::: "memory");
      const fast::Staged sg{sbuf + buf * 4 * ss + t, ss};
      buf ^= 1;
      float2 X, Y, Z;
      fast::decode2_full<G, true>(ww.x, ww.y, F, tab_t, tab_p, X, Y, Z, &sg);
      __stcs(v2 + 3 * i, make_float2(X.x, Y.x));
      __stcs(v2 + 3 * i + 1, make_float2(Z.x, X.y));
      __stcs(v2 + 3 * i + 2, make_float2(Y.y, Z.y));
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
  } else {
  ulonglong2 nw = i0 < n2 ? __ldcs(w2 + i0) : make_ulonglong2(0ull, 0ull);  // next words
  for (int64_t i = i0; i < n2; i += stride) {
    const ulonglong2 ww = nw;
    if (i + stride < n2) nw = __ldcs(w2 + i + stride);
    float2 X, Y, Z;
    // no per-code table: phi^ from the shared head table
    fast::decode2_full<G, false>(ww.x, ww.y, F, tab_t, tab_p, X, Y, Z);
    __stcs(v2 + 3 * i, make_float2(X.x, Y.x));
    __stcs(v2 + 3 * i + 1, make_float2(Z.x, X.y));
    __stcs(v2 + 3 * i + 2, make_float2(Y.y, Z.y));
  }
  }
  if ((n & 1) && blockIdx.x == 0 && threadIdx.x == 0) {
    const int64_t i = n - 1;
    const float3 v = decode_word<G::MAP>(w[i], F, tab_t, tab_p);
    xyz[3 * i] = v.x;
    xyz[3 * i + 1] = v.y;
    xyz[3 * i + 2] = v.z;
  }
}

// v_out = encode(fmaf(dt, f, v)); m_out = encode(rho * v_new) (if requested).
template <class G>
__global__ void __launch_bounds__(256, 3) k_update_fast(const __grid_constant__ DevFormat F, float dt,
                                                     const uint64_t *v, const uint64_t *f,
                                                     const float *__restrict__ rho,
                                                     uint64_t *v_out, uint64_t *m_out, int64_t n) {
  IVC_FAST_TABLES(F, G);
  const bool want_m = (rho != nullptr) && (m_out != nullptr);
  const int64_t n2 = n >> 1;
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const ulonglong2 *v2 = reinterpret_cast<const ulonglong2 *>(v);
  const ulonglong2 *f2 = reinterpret_cast<const ulonglong2 *>(f);
  ulonglong2 *o2 = reinterpret_cast<ulonglong2 *>(v_out);
  ulonglong2 *m2 = reinterpret_cast<ulonglong2 *>(m_out);
  fast::WarpQueue wq = fast::warp_queue(IVC_FAST_QUEUE(F, G));
  ulonglong2 nv = make_ulonglong2(0ull, 0ull), nf = nv;  // next iteration's words
  if (warp * 32 + lane < n2) {
    nv = __ldcs(v2 + warp * 32 + lane);
    nf = __ldcs(f2 + warp * 32 + lane);
  }
  for (int64_t base = warp * 32; base < n2; base += nwarps * 32) {
    const int64_t i = base + lane;
    const bool act = i < n2;
    const ulonglong2 wv = nv, wf = nf;
    if (i + nwarps * 32 < n2) {
      nv = __ldcs(v2 + i + nwarps * 32);
      nf = __ldcs(f2 + i + nwarps * 32);
    }
    float2 ux, uy, uz, gx, gy, gz;
    fast::decode2_full<G>(wv.x, wv.y, F, tab_t, tab_p, ux, uy, uz);
    fast::decode2_full<G>(wf.x, wf.y, F, tab_t, tab_p, gx, gy, gz);
    const float2 sx = fast::fma2(fast::bc(dt), gx, ux);
    const float2 sy = fast::fma2(fast::bc(dt), gy, uy);
    const float2 sz = fast::fma2(fast::bc(dt), gz, uz);
    fast::Est2 est;
    const fast::Enc2 e = fast::encode2<G>(sx, sy, sz, F, tab_t, tab_p, &est);
    if (act) __stcs(o2 + i, make_ulonglong2(e.w0, e.w1));
    fast::push2<G>(wq, act, e, sx, sy, sz, v_out + 2 * i, F, tab_t, tab_p);
    if (want_m) {
      const float2 q = act ? make_float2(__ldcs(rho + 2 * i), __ldcs(rho + 2 * i + 1))
                           : make_float2(0.0f, 0.0f);
      const float2 mx = fast::mul2(q, sx), my = fast::mul2(q, sy), mz = fast::mul2(q, sz);
      // m = RN(rho v) points where v does (rho > 0): v's angle estimates
      // serve m, with the ambiguity band widened by the rounding of rho v
      const bool f0 = !(q.x > 0.0f && q.x < INFINITY) || (e.pend0 & 4u) != 0u;
      const bool f1 = !(q.y > 0.0f && q.y < INFINITY) || (e.pend1 & 4u) != 0u;
      const fast::Enc2 em = fast::encode2<G, true>(mx, my, mz, F, tab_t, tab_p, &est, f0, f1);
      if (act) __stcs(m2 + i, make_ulonglong2(em.w0, em.w1));
      fast::push2<G>(wq, act, em, mx, my, mz, m_out + 2 * i, F, tab_t, tab_p);
    }
  }
  fast::drain<G>(wq, F, tab_t, tab_p);
  if ((n & 1) && blockIdx.x == 0 && threadIdx.x == 0) {
    uint32_t flags = 0;
    const int64_t i = n - 1;
    const float3 vv = decode_word<G::MAP>(v[i], F, tab_t, tab_p);
    const float3 ff = decode_word<G::MAP>(f[i], F, tab_t, tab_p);
    const float sx = fmaf(dt, ff.x, vv.x), sy = fmaf(dt, ff.y, vv.y), sz = fmaf(dt, ff.z, vv.z);
    v_out[i] = encode_vec<G::MAP>(sx, sy, sz, F, tab_t, tab_p, flags);
    if (want_m) {
      const float q = rho[i];
      m_out[i] = encode_vec<G::MAP>(q * sx, q * sy, q * sz, F, tab_t, tab_p, flags);
    }
  }
}

// ------------------------------------------------------------------- batched

// Persistent kernel: blocks pull tiles from a device counter; the loop is
// bounded by the tile count (every pull advances the counter), and reports
// IVC_ERR_TIMEOUT in the plan status if the bound is ever reached.
template <int MAP, int OP>
__global__ void __launch_bounds__(256) k_batched(const __grid_constant__ DevFormat F,
                                                 const __grid_constant__ PlanDev P) {
  IVC_TABLES(F, MAP);
  __shared__ long long s_tile;
  uint32_t flags = 0;
  bool done = false;
  for (int64_t iter = 0; iter <= P.total_tiles; ++iter) {
    if (threadIdx.x == 0) s_tile = (long long)atomicAdd(P.counter, 1ull);
    __syncthreads();
    const int64_t tile = s_tile;
    __syncthreads();
    if (tile >= P.total_tiles) {
      done = true;
      break;
    }
    // field of this tile: last f with tile_start[f] <= tile
    int lo = 0, hi = P.nfields;  // tile_start[lo] <= tile < tile_start[hi]
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (P.tile_start[mid] <= tile) lo = mid; else hi = mid;
    }
    const FieldDesc fd = P.fields[lo];
    const int64_t start = (tile - P.tile_start[lo]) * (int64_t)P.tile;
    // a work-list entry that names no range inside its field (a plan whose
    // workspace was overwritten) is skipped and reported
    if (start < 0 || start >= fd.n) {
      if (threadIdx.x == 0) atomicExch(P.status, (int)IVC_ERR_ARG);
      continue;
    }
    const int64_t len = min((int64_t)P.tile, fd.n - start);
    const uint64_t *a = fd.a + start;
    const uint64_t *b = (OP == IVC_OP_ADD ? fd.b : fd.c) + start;
    uint64_t *c = fd.c + start;
    const bool vec2 = ((reinterpret_cast<uintptr_t>(a) | reinterpret_cast<uintptr_t>(b) |
                        reinterpret_cast<uintptr_t>(c)) & 15u) == 0;
    if (OP == IVC_OP_ADD)
      fused_range<MAP>(a, b, c, len, vec2, threadIdx.x, blockDim.x, OpAdd{}, F, tab_t, tab_p,
                       flags);
    else
      fused_range<MAP>(a, b, c, len, vec2, threadIdx.x, blockDim.x, OpAxpy{fd.alpha}, F, tab_t,
                       tab_p, flags);
  }
  if (!done && threadIdx.x == 0) atomicExch(P.status, (int)IVC_ERR_TIMEOUT);
}

// Batched persistent kernel on the primary-layout fast path (tiles of an
// even number of words; 16-byte aligned fields use the packed loop).
template <int OP, class G>
__global__ void __launch_bounds__(256) k_batched_fast(const __grid_constant__ DevFormat F,
                                                      const __grid_constant__ PlanDev P) {
  IVC_FAST_TABLES(F, G);
  __shared__ long long s_tile;
  uint32_t flags = 0;
  bool done = false;
  for (int64_t iter = 0; iter <= P.total_tiles; ++iter) {
    if (threadIdx.x == 0) s_tile = (long long)atomicAdd(P.counter, 1ull);
    __syncthreads();
    const int64_t tile = s_tile;
    __syncthreads();
    if (tile >= P.total_tiles) {
      done = true;
      break;
    }
    int lo = 0, hi = P.nfields;
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (P.tile_start[mid] <= tile) lo = mid; else hi = mid;
    }
    const FieldDesc fd = P.fields[lo];
    const int64_t start = (tile - P.tile_start[lo]) * (int64_t)P.tile;
    // a work-list entry that names no range inside its field (a plan whose
    // workspace was overwritten) is skipped and reported
    if (start < 0 || start >= fd.n) {
      if (threadIdx.x == 0) atomicExch(P.status, (int)IVC_ERR_ARG);
      continue;
    }
    const int64_t len = min((int64_t)P.tile, fd.n - start);
    const uint64_t *a = fd.a + start;
    const uint64_t *b = (OP == IVC_OP_ADD ? fd.b : fd.c) + start;
    uint64_t *c = fd.c + start;
    const bool vec2 = ((reinterpret_cast<uintptr_t>(a) | reinterpret_cast<uintptr_t>(b) |
                        reinterpret_cast<uintptr_t>(c)) & 15u) == 0;
    if (vec2) {
      fused_fast_range<OP, G>(a, b, c, len, threadIdx.x >> 5, blockDim.x >> 5, threadIdx.x & 31,
                           fd.alpha, F, tab_t, tab_p, IVC_FAST_QUEUE(F, G));
    } else if (OP == IVC_OP_ADD) {
      fused_range<G::MAP>(a, b, c, len, false, threadIdx.x, blockDim.x, OpAdd{}, F, tab_t,
                          tab_p, flags);
    } else {
      fused_range<G::MAP>(a, b, c, len, false, threadIdx.x, blockDim.x, OpAxpy{fd.alpha}, F,
                          tab_t, tab_p, flags);
    }
  }
  if (!done && threadIdx.x == 0) atomicExch(P.status, (int)IVC_ERR_TIMEOUT);
}

// Tiles per field and their prefix sums (one block; nfields is small).
__global__ void k_tile_scan(const FieldDesc *fields, int nfields, int tile, int64_t *tile_start) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    int64_t acc = 0;
    for (int f = 0; f < nfields; ++f) {
      tile_start[f] = acc;
      const int64_t n = fields[f].n > 0 ? fields[f].n : 0;
      acc += (n + tile - 1) / tile;
    }
    tile_start[nfields] = acc;
  }
}

// ------------------------------------------------------------------ launchers

size_t table_smem_bytes(const DevFormat &F, int map) {
  return map == MAP_TANH ? 0 : (size_t)(F.nent_t + F.nent_p) * sizeof(TabEntry);
}

size_t kernel_smem_bytes(const DevFormat &F, int map, int kind, int block) {
  const bool queue = kind == K_ADD_FAST || kind == K_AXPY_FAST || kind == K_UPDATE_FAST ||
                     kind == K_BATCH_ADD_FAST || kind == K_BATCH_AXPY_FAST ||
                     kind == K_COMPRESS_FAST;
  const bool fastk = queue || kind == K_DECOMPRESS_FAST;
  // the fast kernels of the tanh map stage the encoder's node tables
  const size_t tabs = (fastk && map == MAP_TANH)
                          ? (size_t)(F.nest_t + F.nest_p) * sizeof(TabEntry)
                          : table_smem_bytes(F, map);
  // the tanh map's fused add / axpy stage their decoder's table entries (two
  // buffers of 8 16-byte slots per thread)
  const bool staged = (kind == K_ADD_FAST || kind == K_AXPY_FAST) && map == MAP_TANH;
  const bool dstaged = kind == K_DECOMPRESS_FAST && map != MAP_TANH && F.phi_tab != nullptr;
  return tabs + (queue ? (size_t)(block / 32) * fast::kQueueCap * sizeof(fast::PendItem) : 0) +
         (staged ? (size_t)block * 16 * 16 : 0) + (dstaged ? (size_t)block * 8 * 16 : 0);
}

#define IVC_DISPATCH_MAP(map, KERNEL, ...)                                                    \
  switch (map) {                                                                              \
    case MAP_UNIFORM: KERNEL<MAP_UNIFORM><<<s.grid, s.block, s.smem, st>>>(__VA_ARGS__); break; \
    case MAP_TANH: KERNEL<MAP_TANH><<<s.grid, s.block, s.smem, st>>>(__VA_ARGS__); break;       \
    default: KERNEL<MAP_FRACSPLIT><<<s.grid, s.block, s.smem, st>>>(__VA_ARGS__); break;       \
  }                                                                                           \
  return cudaGetLastError()

cudaError_t launch_compress(int map, const DevFormat &F, const float *xyz, int layout, int64_t ld,
                            int64_t n, uint64_t *w, ivc_counts *counts, const LaunchShape &s,
                            cudaStream_t st) {
  IVC_DISPATCH_MAP(map, k_compress, F, xyz, layout, ld, n, w, counts);
}

cudaError_t launch_decompress(int map, const DevFormat &F, const uint64_t *w, int64_t n,
                              float *xyz, int layout, int64_t ld, const LaunchShape &s,
                              cudaStream_t st) {
  IVC_DISPATCH_MAP(map, k_decompress, F, w, n, xyz, layout, ld);
}

cudaError_t launch_compress_exact(int map, const DevFormat &F, const float *xyz, int64_t n,
                                  uint64_t *w, ivc_counts *counts, const LaunchShape &s,
                                  cudaStream_t st) {
  switch (map) {
    case MAP_UNIFORM:
      k_compress<MAP_UNIFORM, true><<<s.grid, s.block, s.smem, st>>>(F, xyz, IVC_AOS, 0, n, w,
                                                                     counts);
      break;
    case MAP_TANH:
      k_compress<MAP_TANH, true><<<s.grid, s.block, s.smem, st>>>(F, xyz, IVC_AOS, 0, n, w, counts);
      break;
    default:
      k_compress<MAP_FRACSPLIT, true><<<s.grid, s.block, s.smem, st>>>(F, xyz, IVC_AOS, 0, n, w,
                                                                       counts);
      break;
  }
  return cudaGetLastError();
}

cudaError_t launch_decompress_exact(int map, const DevFormat &F, const uint64_t *w, int64_t n,
                                    float *xyz, const LaunchShape &s, cudaStream_t st) {
  switch (map) {
    case MAP_UNIFORM:
      k_decompress<MAP_UNIFORM, true><<<s.grid, s.block, s.smem, st>>>(F, w, n, xyz, IVC_AOS, 0);
      break;
    case MAP_TANH:
      k_decompress<MAP_TANH, true><<<s.grid, s.block, s.smem, st>>>(F, w, n, xyz, IVC_AOS, 0);
      break;
    default:
      k_decompress<MAP_FRACSPLIT, true><<<s.grid, s.block, s.smem, st>>>(F, w, n, xyz, IVC_AOS, 0);
      break;
  }
  return cudaGetLastError();
}

cudaError_t launch_add(int map, const DevFormat &F, const uint64_t *a, const uint64_t *b,
                       uint64_t *c, int64_t n, const LaunchShape &s, cudaStream_t st) {
  IVC_DISPATCH_MAP(map, k_add, F, a, b, c, n, s.vec2);
}

cudaError_t launch_axpy(int map, const DevFormat &F, float alpha, const uint64_t *x, uint64_t *y,
                        int64_t n, const LaunchShape &s, cudaStream_t st) {
  IVC_DISPATCH_MAP(map, k_axpy, F, alpha, x, y, n, s.vec2);
}

cudaError_t launch_update(int map, const DevFormat &F, float dt, const uint64_t *v,
                          const uint64_t *f, const float *rho, uint64_t *v_out, uint64_t *m_out,
                          int64_t n, const LaunchShape &s, cudaStream_t st) {
  IVC_DISPATCH_MAP(map, k_update, F, dt, v, f, rho, v_out, m_out, n);
}

// Fast launchers: the layout is read from F (the caller has checked
// fast::fast_geometry()); f receives a value of the layout's type.
// Dynamic shared memory above the 48 KB every kernel may use by default needs
// the kernel's opt-in (the tanh map's fast kernels: node tables and queues).
__host__ inline cudaError_t allow_smem(const void *kernel, size_t smem) {
  if (smem <= 48 * 1024) return cudaSuccess;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

#define IVC_LAUNCH(KERNEL, ...)                                                         \
  do {                                                                                  \
    if (allow_smem((const void *)KERNEL, s.smem) != cudaSuccess) return;                \
    KERNEL<<<s.grid, s.block, s.smem, st>>>(__VA_ARGS__);                               \
  } while (0)

template <class Fn>
cudaError_t with_geo(const DevFormat &F, Fn f) {
  if (fast::is_geo<fast::GeoTanh>(F))
    f(fast::GeoTanh{});
  else if (fast::is_geo<fast::GeoSplit>(F))
    f(fast::GeoSplit{});
  else if (fast::is_geo<fast::GeoL1717>(F))
    f(fast::GeoL1717{});
  else if (fast::is_geo<fast::GeoL1617>(F))
    f(fast::GeoL1617{});
  else
    f(fast::GeoPrimary{});
  return cudaGetLastError();
}

cudaError_t launch_batched(int map, int op, const DevFormat &F, const PlanDev &P,
                           const LaunchShape &s, cudaStream_t st) {
  if (fast::fast_geometry(map, F) != 0) {
    return with_geo(F, [&](auto g) {
      if (op == IVC_OP_ADD)
        IVC_LAUNCH((k_batched_fast<IVC_OP_ADD, decltype(g)>), F, P);
      else
        IVC_LAUNCH((k_batched_fast<IVC_OP_AXPY, decltype(g)>), F, P);
    });
  }
  if (op == IVC_OP_ADD) {
    switch (map) {
      case MAP_UNIFORM: k_batched<MAP_UNIFORM, IVC_OP_ADD><<<s.grid, s.block, s.smem, st>>>(F, P); break;
      case MAP_TANH: k_batched<MAP_TANH, IVC_OP_ADD><<<s.grid, s.block, s.smem, st>>>(F, P); break;
      default: k_batched<MAP_FRACSPLIT, IVC_OP_ADD><<<s.grid, s.block, s.smem, st>>>(F, P); break;
    }
  } else {
    switch (map) {
      case MAP_UNIFORM: k_batched<MAP_UNIFORM, IVC_OP_AXPY><<<s.grid, s.block, s.smem, st>>>(F, P); break;
      case MAP_TANH: k_batched<MAP_TANH, IVC_OP_AXPY><<<s.grid, s.block, s.smem, st>>>(F, P); break;
      default: k_batched<MAP_FRACSPLIT, IVC_OP_AXPY><<<s.grid, s.block, s.smem, st>>>(F, P); break;
    }
  }
  return cudaGetLastError();
}

cudaError_t launch_add_fast(const DevFormat &F, const uint64_t *a, const uint64_t *b, uint64_t *c,
                            int64_t n, const LaunchShape &s, cudaStream_t st) {
  return with_geo(F, [&](auto g) {
    if (F.phi_tab || decltype(g)::MAP == MAP_TANH)
      IVC_LAUNCH((k_fused_fast<IVC_OP_ADD, decltype(g), true>), F, a, b, c, n, 0.0f);
    else  // no per-code phi^ table (the allocation-free entry point)
      IVC_LAUNCH((k_fused_fast<IVC_OP_ADD, decltype(g), false>), F, a, b, c, n, 0.0f);
  });
}

cudaError_t launch_axpy_fast(const DevFormat &F, float alpha, const uint64_t *x, uint64_t *y,
                             int64_t n, const LaunchShape &s, cudaStream_t st) {
  return with_geo(F, [&](auto g) {
    IVC_LAUNCH((k_fused_fast<IVC_OP_AXPY, decltype(g), true>), F, x, y, y, n, alpha);
  });
}

cudaError_t launch_compress_fast(const DevFormat &F, const float *xyz, int64_t n, uint64_t *w,
                                 ivc_counts *counts, const LaunchShape &s, cudaStream_t st) {
  return with_geo(F, [&](auto g) {
    IVC_LAUNCH((k_compress_fast<decltype(g)>), F, xyz, n, w, counts);
  });
}

cudaError_t launch_decompress_fast(const DevFormat &F, const uint64_t *w, int64_t n, float *xyz,
                                   const LaunchShape &s, cudaStream_t st) {
  return with_geo(F, [&](auto g) {
    IVC_LAUNCH((k_decompress_fast<decltype(g)>), F, w, n, xyz);
  });
}

cudaError_t launch_update_fast(const DevFormat &F, float dt, const uint64_t *v, const uint64_t *f,
                               const float *rho, uint64_t *v_out, uint64_t *m_out, int64_t n,
                               const LaunchShape &s, cudaStream_t st) {
  return with_geo(F, [&](auto g) {
    IVC_LAUNCH((k_update_fast<decltype(g)>), F, dt, v, f, rho, v_out, m_out, n);
  });
}

cudaError_t launch_tile_scan(const FieldDesc *fields, int nfields, int tile, int64_t *tile_start,
                             cudaStream_t st) {
  k_tile_scan<<<1, 32, 0, st>>>(fields, nfields, tile, tile_start);
  return cudaGetLastError();
}

template <int MAP>
static const void *kernel_ptr(int kind) {
  using G = std::conditional_t<MAP == MAP_TANH, fast::GeoTanh, fast::GeoPrimary>;
  switch (kind) {
    case K_COMPRESS: return (const void *)k_compress<MAP>;
    case K_DECOMPRESS: return (const void *)k_decompress<MAP>;
    case K_ADD: return (const void *)k_add<MAP>;
    case K_AXPY: return (const void *)k_axpy<MAP>;
    case K_UPDATE: return (const void *)k_update<MAP>;
    case K_BATCH_ADD: return (const void *)k_batched<MAP, IVC_OP_ADD>;
    case K_ADD_FAST: return (const void *)k_fused_fast<IVC_OP_ADD, G, true>;
    case K_AXPY_FAST: return (const void *)k_fused_fast<IVC_OP_AXPY, G, true>;
    case K_UPDATE_FAST: return (const void *)k_update_fast<G>;
    case K_BATCH_ADD_FAST: return (const void *)k_batched_fast<IVC_OP_ADD, G>;
    case K_COMPRESS_FAST: return (const void *)k_compress_fast<G>;
    case K_DECOMPRESS_FAST: return (const void *)k_decompress_fast<G>;
    case K_BATCH_AXPY_FAST: return (const void *)k_batched_fast<IVC_OP_AXPY, G>;
    default: return (const void *)k_batched<MAP, IVC_OP_AXPY>;
  }
}

int occupancy(int map, int kind, int block, size_t smem) {
  const void *k = map == MAP_UNIFORM ? kernel_ptr<MAP_UNIFORM>(kind)
                  : map == MAP_TANH  ? kernel_ptr<MAP_TANH>(kind)
                                     : kernel_ptr<MAP_FRACSPLIT>(kind);
  int nb = 0;
  if (allow_smem(k, smem) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, block, smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return nb;
}

}  // namespace ivc
