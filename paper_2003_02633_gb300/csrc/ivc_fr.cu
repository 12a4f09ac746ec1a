// Flux-reconstruction steps 5-11 of Table fr_nse (Sec. 4) with the gradient,
// metric, normal and flux tensors held as compressed rows (Eq. eulerF: every
// row of a tensor is one 3-vector, compressed on its own), and the same steps
// on FP32 rows as the baseline.  Step 10 is Algorithm 1 (ivc_fdiv.cu).
//
//   5  gradient      w^s (scalars)             -> grad w^s (rows)
//   6  correction    grad w^s, jumps at faces  -> grad w^c (rows)
//   7  interpolation grad w^c                  -> grad w^f (rows at faces)
//   8  common viscous flux (BR1) at faces, both sides' rows -> n.(F_inv - F_vis)
//   9  flux          q^s, grad w^s, metric rows -> F^s (rows)
//   11 correction    F^s, interface flux       -> F^fc
//
// Layout (element index fastest, one leading dimension ld >= ne for every
// array of a call): scalars of point k, variable v at [(k nv + v) ld + e];
// compressed rows at the same index; FP32 rows with component c at
// [((c npts + k) nv + v) ld + e].
//
// GB300 layout of the work: a block of 8 warps owns a tile of 64 elements
// (lane and lane + 32, so that every warp-wide load or store is two runs of
// 32 consecutive elements) and one variable or one point at a time.  The
// element-local contractions (5, 7, 11) first stage the tile's inputs in
// shared memory as FP32 (decoding each compressed row once), then evaluate
// the tensor-product operators in sum-factorised form (q terms per output, the
// 1-D basis in the kernel's parameter space) and encode two outputs per
// thread (packed fast path, exact tests deferred to the per-warp queue).  The
// pointwise step 6 decodes, computes in FP32 and encodes in registers; the
// pointwise steps 8 and 9 stage compressed rows in per-thread shared-memory
// slots (k_fr_commonvis_w, k_fr_flux_w) and FP32 rows in registers.
#include "ivc_decode_poles.cuh"
#include "ivc_internal.h"

namespace ivc {
namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kTile = 64;  // elements per tile
constexpr int kMaxQ = 4;   // points per axis (degree <= 3)

struct FrBasisDev {
  int q;
  float dm[kMaxQ][kMaxQ];  // dm[i][a] = l_a'(xi_i)
  float lm[kMaxQ], lp[kMaxQ], gl[kMaxQ], gr[kMaxQ];
  // Index tables, so that the kernels' loops over points and flux points
  // divide nothing by q.  Flux point f: first solution point of its line
  // (bits 0-7), the line's point stride (8-15), side (16), axis (17-18).
  // Solution point k: its indices i, j, l along the three axes (2 bits each,
  // bits 0-5) and, per axis c, the flux point of side 0 on its line (7 bits
  // each from bit 6 + 7c).
  int fdesc[6 * kMaxQ * kMaxQ];
  int pdesc[kMaxQ * kMaxQ * kMaxQ];
};

struct FrGasDev {
  float gamma, mu, kappa;  // kappa = mu gamma / ((gamma - 1) Pr)
};

// Dynamic shared memory: tables | per-warp queues | staging buffer.
struct FrSmem {
  int off_queue, off_stage;
};

// ------------------------------------------------------------ row codecs

// Queues the pending words of an encoded pair written at d0 and d1 (lanes
// with v0 / v1 false queue nothing) and resolves full batches.  All lanes of
// the warp call it.
template <class G>
__device__ __forceinline__ void push_pair(fast::WarpQueue &wq, bool v0, bool v1,
                                          const fast::Enc2 &e, float2 x, float2 y, float2 z,
                                          uint64_t *d0, uint64_t *d1, const DevFormat &F,
                                          const TabEntry *tab_t, const TabEntry *tab_p) {
  const uint32_t p0 = v0 ? e.pend0 : 0u, p1 = v1 ? e.pend1 : 0u;
  const unsigned b0 = __ballot_sync(0xffffffffu, p0 != 0u);
  const unsigned b1 = __ballot_sync(0xffffffffu, p1 != 0u);
  if ((b0 | b1) == 0u) return;
  const unsigned lt = (1u << (threadIdx.x & 31)) - 1u;
  int slot = wq.count + __popc(b0 & lt) + __popc(b1 & lt);
  if (p0) {
    wq.q[slot++] = fast::PendItem{d0, x.x, y.x, z.x, e.hi0, e.nt0, (uint32_t)e.np0 | (p0 << 29)};
  }
  if (p1) {
    wq.q[slot] = fast::PendItem{d1, x.y, y.y, z.y, e.hi1, e.nt1, (uint32_t)e.np1 | (p1 << 29)};
  }
  wq.count += __popc(b0) + __popc(b1);
  while (wq.count >= 32) {
    __syncwarp();
    fast::resolve_item<G>(wq.q + wq.count - 32 + (threadIdx.x & 31), F, tab_t, tab_p);
    wq.count -= 32;
    __syncwarp();
  }
}

// Compressed rows, fast path of layout G: packed decode and encode; the rows
// are decoded in plain FP32 (within 22 2^-24 relative of the canonical decoded
// values, which these FP32 steps need only to within their own rounding).
template <class G>
struct FastRows {
  using T = uint64_t;
  static constexpr bool kWords = true;
  static constexpr bool kQueue = true;
  const DevFormat &F;
  const TabEntry *tab_t, *tab_p;
  fast::WarpQueue wq;

  struct Raw {
    uint64_t w0, w1;
  };
  __device__ Raw fetch2(const T *src, int64_t i0, int64_t i1, bool v0, bool v1, int64_t) const {
    return Raw{v0 ? __ldg(src + i0) : 0ull, v1 ? __ldg(src + i1) : 0ull};
  }
  __device__ void decode_raw(const Raw &r, float2 &X, float2 &Y, float2 &Z) const {
    fast::decode2_f32<G>(r.w0, r.w1, F, tab_t, tab_p, X, Y, Z);
  }
  __device__ void load2(const T *src, int64_t i0, int64_t i1, bool v0, bool v1, int64_t cs,
                        float2 &X, float2 &Y, float2 &Z) const {
    decode_raw(fetch2(src, i0, i1, v0, v1, cs), X, Y, Z);
  }
  __device__ void store2(T *dst, int64_t i0, int64_t i1, bool v0, bool v1, int64_t, float2 X,
                         float2 Y, float2 Z) {
    const fast::Enc2 e = fast::encode2<G>(X, Y, Z, F, tab_t, tab_p);
    if (v0) dst[i0] = e.w0;
    if (v1) dst[i1] = e.w1;
    push_pair<G>(wq, v0, v1, e, X, Y, Z, dst + i0, dst + i1, F, tab_t, tab_p);
  }
  __device__ void finish() { fast::drain<G>(wq, F, tab_t, tab_p); }
};

// Compressed rows of any layout and map through the generic decoder and
// encoder, one row at a time.
template <int MAP_>
struct GenericRows {
  using T = uint64_t;
  static constexpr bool kWords = true;
  static constexpr bool kQueue = false;
  static constexpr int MAP = MAP_;
  const DevFormat &F;
  const TabEntry *tab_t, *tab_p;

  struct Raw {
    uint64_t w0, w1;  // 0 (the zero vector) for an absent element
  };
  __device__ Raw fetch2(const T *src, int64_t i0, int64_t i1, bool v0, bool v1, int64_t) const {
    return Raw{v0 ? __ldg(src + i0) : 0ull, v1 ? __ldg(src + i1) : 0ull};
  }
  __device__ void decode_raw(const Raw &r, float2 &X, float2 &Y, float2 &Z) const {
    const float3 a = decode_word<MAP>(r.w0, F, tab_t, tab_p);
    const float3 b = decode_word<MAP>(r.w1, F, tab_t, tab_p);
    X = make_float2(a.x, b.x);
    Y = make_float2(a.y, b.y);
    Z = make_float2(a.z, b.z);
  }
  __device__ void load2(const T *src, int64_t i0, int64_t i1, bool v0, bool v1, int64_t cs,
                        float2 &X, float2 &Y, float2 &Z) const {
    decode_raw(fetch2(src, i0, i1, v0, v1, cs), X, Y, Z);
  }
  __device__ void store2(T *dst, int64_t i0, int64_t i1, bool v0, bool v1, int64_t, float2 X,
                         float2 Y, float2 Z) {
    uint32_t flags = 0;
    if (v0) dst[i0] = encode_vec<MAP>(X.x, Y.x, Z.x, F, tab_t, tab_p, flags);
    if (v1) dst[i1] = encode_vec<MAP>(X.y, Y.y, Z.y, F, tab_t, tab_p, flags);
  }
  __device__ void finish() {}
};

// FP32 rows: component c at offset c * cs from the row's index.
struct F32Rows {
  using T = float;
  static constexpr bool kWords = false;
  static constexpr bool kQueue = false;

  struct Raw {
    float2 x, y, z;
  };
  __device__ Raw fetch2(const T *src, int64_t i0, int64_t i1, bool v0, bool v1,
                        int64_t cs) const {
    return Raw{make_float2(v0 ? __ldg(src + i0) : 0.0f, v1 ? __ldg(src + i1) : 0.0f),
               make_float2(v0 ? __ldg(src + i0 + cs) : 0.0f, v1 ? __ldg(src + i1 + cs) : 0.0f),
               make_float2(v0 ? __ldg(src + i0 + 2 * cs) : 0.0f,
                           v1 ? __ldg(src + i1 + 2 * cs) : 0.0f)};
  }
  __device__ void decode_raw(const Raw &r, float2 &X, float2 &Y, float2 &Z) const {
    X = r.x;
    Y = r.y;
    Z = r.z;
  }
  __device__ void load2(const T *src, int64_t i0, int64_t i1, bool v0, bool v1, int64_t cs,
                        float2 &X, float2 &Y, float2 &Z) const {
    decode_raw(fetch2(src, i0, i1, v0, v1, cs), X, Y, Z);
  }
  __device__ void store2(T *dst, int64_t i0, int64_t i1, bool v0, bool v1, int64_t cs, float2 X,
                         float2 Y, float2 Z) {
    if (v0) {
      dst[i0] = X.x;
      dst[i0 + cs] = Y.x;
      dst[i0 + 2 * cs] = Z.x;
    }
    if (v1) {
      dst[i1] = X.y;
      dst[i1 + cs] = Y.y;
      dst[i1 + 2 * cs] = Z.y;
    }
  }
  __device__ void finish() {}
};

// Codec objects per kernel: tables staged in shared memory for word codecs.
template <class C>
struct CodecOf;

template <class G>
struct CodecOf<FastRows<G>> {
  __device__ static FastRows<G> make(const DevFormat &F, unsigned char *smem, const FrSmem &L) {
    TabEntry *tab = reinterpret_cast<TabEntry *>(smem);
    stage_tables<G::MAP>(F, tab);
    return FastRows<G>{F, tab, tab + F.nent_t, fast::warp_queue(smem + L.off_queue)};
  }
};

template <int MAP>
struct CodecOf<GenericRows<MAP>> {
  __device__ static GenericRows<MAP> make(const DevFormat &F, unsigned char *smem,
                                          const FrSmem &) {
    TabEntry *tab = reinterpret_cast<TabEntry *>(smem);
    stage_tables<MAP>(F, tab);
    return GenericRows<MAP>{F, tab, tab + (MAP == MAP_TANH ? 0 : F.nent_t)};
  }
};

template <>
struct CodecOf<F32Rows> {
  __device__ static F32Rows make(const DevFormat &, unsigned char *, const FrSmem &) {
    return F32Rows{};
  }
};

// ------------------------------------------------------------ index helpers

// The definitions of the point and flux-point numbering; the host builds the
// kernels' index tables (FrBasisDev::fdesc, pdesc) from them.
__host__ __device__ __forceinline__ void point_ijk(int k, int q, int ijk[3]) {
  ijk[0] = k % q;
  ijk[1] = (k / q) % q;
  ijk[2] = k / (q * q);
}

__host__ __device__ __forceinline__ int point_of(const int ijk[3], int q) {
  return (ijk[2] * q + ijk[1]) * q + ijk[0];
}

// Flux point f -> face axis c, side s and the indices along the other axes.
__host__ __device__ __forceinline__ void face_of(int f, int q, int &c, int &s, int ijk[3]) {
  const int face = f / (q * q), ab = f % (q * q);
  c = face >> 1;
  s = face & 1;
  const int o0 = c == 0 ? 1 : 0, o1 = c == 2 ? 1 : 2;
  ijk[o0] = ab % q;
  ijk[o1] = ab / q;
  ijk[c] = 0;
}

// Flux point of side s of axis c on the line of solution point ijk.
__host__ __device__ __forceinline__ int flux_point(int c, int s, const int ijk[3], int q) {
  const int o0 = c == 0 ? 1 : 0, o1 = c == 2 ? 1 : 2;
  return (2 * c + s) * q * q + ijk[o1] * q + ijk[o0];
}

// The line of solution points through flux point f, from the table.
struct FaceLine {
  int base, stride, side, axis;
};

__device__ __forceinline__ FaceLine face_line(const FrBasisDev &B, int f) {
  const int d = B.fdesc[f];
  return FaceLine{d & 0xff, (d >> 8) & 0xff, (d >> 16) & 1, (d >> 17) & 3};
}

// Index of solution point k along axis c, and the flux point of side 0 on
// its line along c, from the table entry pd = B.pdesc[k].
__device__ __forceinline__ int pd_index(int pd, int c) { return (pd >> (2 * c)) & 3; }
__device__ __forceinline__ int pd_flux0(int pd, int c) { return (pd >> (6 + 7 * c)) & 0x7f; }

// (tile, sub) = divmod(it, nsub) for it = first, first + step, ... (a
// per-warp or per-block item loop), advanced without a 64-bit division per
// item; tile < ntiles exactly while it < ntiles * nsub.
struct ItemWalk {
  int64_t tile, dtile;
  int sub, dsub, nsub;
  __device__ ItemWalk(int64_t first, int64_t step, int n) : nsub(n) {
    tile = first / n;
    sub = (int)(first - tile * n);
    dtile = step / n;
    dsub = (int)(step - dtile * n);
  }
  __device__ void next() {
    tile += dtile;
    sub += dsub;
    if (sub >= nsub) {
      sub -= nsub;
      ++tile;
    }
  }
};

// ------------------------------------------------------------ step 5

// grad w (rows at the solution points) of the scalars w.
template <class C>
__global__ void __launch_bounds__(kThreads) k_fr_grad(const __grid_constant__ DevFormat F,
                                                      const __grid_constant__ FrBasisDev B,
                                                      FrSmem L, const float *__restrict__ w,
                                                      int64_t ne, int64_t ld, int nv,
                                                      typename C::T *out) {
  extern __shared__ __align__(16) unsigned char smem[];
  C codec = CodecOf<C>::make(F, smem, L);
  float *sw = reinterpret_cast<float *>(smem + L.off_stage);  // [ns][64]
  const int q = B.q, ns = q * q * q;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t ntiles = (ne + kTile - 1) / kTile;
  const int64_t items = ntiles * nv;
  const int64_t cs = (int64_t)ns * nv * ld;
  for (int64_t it = blockIdx.x; it < items; it += gridDim.x) {
    const int64_t e0 = (it / nv) * kTile;
    const int v = (int)(it % nv);
    const int64_t ea = e0 + lane, eb = e0 + lane + 32;
    const bool va = ea < ne, vb = eb < ne;
    for (int k = warp; k < ns; k += kWarps) {
      const float *row = w + ((int64_t)k * nv + v) * ld;
      sw[k * kTile + lane] = va ? __ldg(row + ea) : 0.0f;
      sw[k * kTile + lane + 32] = vb ? __ldg(row + eb) : 0.0f;
    }
    __syncthreads();
    for (int k = warp; k < ns; k += kWarps) {
      const int pd = B.pdesc[k];
      float2 g[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const int ic = pd_index(pd, c);
        const int stride = c == 0 ? 1 : (c == 1 ? q : q * q);
        const float *r = sw + (k - ic * stride) * kTile + lane;
        float ga = 0.0f, gb = 0.0f;
#pragma unroll
        for (int a = 0; a < kMaxQ; ++a) {
          if (a < q) {
            const float d = B.dm[ic][a];
            ga = fmaf(d, r[a * stride * kTile], ga);
            gb = fmaf(d, r[a * stride * kTile + 32], gb);
          }
        }
        g[c] = make_float2(ga, gb);
      }
      const int64_t idx = ((int64_t)k * nv + v) * ld;
      codec.store2(out, idx + ea, idx + eb, va, vb, cs, g[0], g[1], g[2]);
    }
    __syncthreads();
  }
  codec.finish();
}

// ------------------------------------------------------------ step 6

// grad w^c = grad w^s + g_L'(xi) dw(left face) + g_R'(xi) dw(right face),
// axis by axis; G == Gc is allowed.
template <class C>
__global__ void __launch_bounds__(kThreads) k_fr_correct(const __grid_constant__ DevFormat F,
                                                         const __grid_constant__ FrBasisDev B,
                                                         FrSmem L, const typename C::T *G,
                                                         const float *__restrict__ dw,
                                                         int64_t ne, int64_t ld, int nv,
                                                         typename C::T *Gc) {
  extern __shared__ __align__(16) unsigned char smem[];
  C codec = CodecOf<C>::make(F, smem, L);
  float *sd = reinterpret_cast<float *>(smem + L.off_stage);  // [nf][64]
  const int q = B.q, ns = q * q * q, nf = 6 * q * q;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t ntiles = (ne + kTile - 1) / kTile;
  const int64_t items = ntiles * nv;
  const int64_t cs = (int64_t)ns * nv * ld;
  for (int64_t it = blockIdx.x; it < items; it += gridDim.x) {
    const int64_t e0 = (it / nv) * kTile;
    const int v = (int)(it % nv);
    const int64_t ea = e0 + lane, eb = e0 + lane + 32;
    const bool va = ea < ne, vb = eb < ne;
    for (int f = warp; f < nf; f += kWarps) {
      const float *row = dw + ((int64_t)f * nv + v) * ld;
      sd[f * kTile + lane] = va ? __ldg(row + ea) : 0.0f;
      sd[f * kTile + lane + 32] = vb ? __ldg(row + eb) : 0.0f;
    }
    // the gradient rows are fetched one point ahead (the first before the barrier)
    typename C::Raw cur{};
    if (warp < ns) {
      const int64_t idx = ((int64_t)warp * nv + v) * ld;
      cur = codec.fetch2(G, idx + ea, idx + eb, va, vb, cs);
    }
    __syncthreads();
    for (int k = warp; k < ns; k += kWarps) {
      const int pd = B.pdesc[k];
      const int64_t idx = ((int64_t)k * nv + v) * ld;
      typename C::Raw nxt = cur;
      if (k + kWarps < ns) {
        const int64_t idn = ((int64_t)(k + kWarps) * nv + v) * ld;
        nxt = codec.fetch2(G, idn + ea, idn + eb, va, vb, cs);
      }
      float2 g[3];
      codec.decode_raw(cur, g[0], g[1], g[2]);
      cur = nxt;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const int fl = pd_flux0(pd, c), fr = fl + q * q;
        const float wl = B.gl[pd_index(pd, c)], wr = B.gr[pd_index(pd, c)];
        g[c].x = fmaf(wr, sd[fr * kTile + lane], fmaf(wl, sd[fl * kTile + lane], g[c].x));
        g[c].y = fmaf(wr, sd[fr * kTile + lane + 32],
                      fmaf(wl, sd[fl * kTile + lane + 32], g[c].y));
      }
      codec.store2(Gc, idx + ea, idx + eb, va, vb, cs, g[0], g[1], g[2]);
    }
    __syncthreads();
  }
  codec.finish();
}

// ------------------------------------------------------------ steps 7, 11

// Stages the tile's rows of variable v at the ns solution points, decoded, as
// [k][c][64] FP32.  AHEAD issues all of a warp's loads before its first decode
// (faster where the registers it takes do not cost occupancy: the compressed
// interpolation; slower for the correction kernel and for FP32 rows, measured).
template <bool AHEAD, class C>
__device__ __forceinline__ void stage_rows(const C &codec, const typename C::T *X, float *sx,
                                           int ns, int nv, int v, int64_t ld, int64_t e0,
                                           int64_t ne, int64_t cs) {
  constexpr int kPer = (kMaxQ * kMaxQ * kMaxQ + kWarps - 1) / kWarps;  // points per warp
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t ea = e0 + lane, eb = e0 + lane + 32;
  const bool va = ea < ne, vb = eb < ne;
  if constexpr (!AHEAD) {
    for (int k = warp; k < ns; k += kWarps) {
      const int64_t idx = ((int64_t)k * nv + v) * ld;
      float2 X0, Y0, Z0;
      codec.load2(X, idx + ea, idx + eb, va, vb, cs, X0, Y0, Z0);
      float *s = sx + k * 3 * kTile;
      s[lane] = X0.x;
      s[lane + 32] = X0.y;
      s[kTile + lane] = Y0.x;
      s[kTile + lane + 32] = Y0.y;
      s[2 * kTile + lane] = Z0.x;
      s[2 * kTile + lane + 32] = Z0.y;
    }
  } else {
    // all of this warp's loads first, then the decodes
    typename C::Raw raw[kPer];
#pragma unroll
    for (int i = 0; i < kPer; ++i) {
      const int k = warp + i * kWarps;
      if (k < ns) {
        const int64_t idx = ((int64_t)k * nv + v) * ld;
        raw[i] = codec.fetch2(X, idx + ea, idx + eb, va, vb, cs);
      }
    }
#pragma unroll
    for (int i = 0; i < kPer; ++i) {
      const int k = warp + i * kWarps;
      if (k < ns) {
        float2 X0, Y0, Z0;
        codec.decode_raw(raw[i], X0, Y0, Z0);
        float *s = sx + k * 3 * kTile;
        s[lane] = X0.x;
        s[lane + 32] = X0.y;
        s[kTile + lane] = Y0.x;
        s[kTile + lane + 32] = Y0.y;
        s[2 * kTile + lane] = Z0.x;
        s[2 * kTile + lane + 32] = Z0.y;
      }
    }
  }
}

// Value on face line fl of component comp of the staged rows (q-term sum
// along the face's axis), for tile elements lane and lane + 32.
__device__ __forceinline__ float2 line_value(const float *sx, const FrBasisDev &B,
                                             const FaceLine &fl, int comp, int lane) {
  const float *r = sx + (fl.base * 3 + comp) * kTile + lane;
  const int step = fl.stride * 3 * kTile;
  float a = 0.0f, b = 0.0f;
#pragma unroll
  for (int i = 0; i < kMaxQ; ++i) {
    if (i < B.q) {
      const float l = fl.side ? B.lp[i] : B.lm[i];
      a = fmaf(l, r[i * step], a);
      b = fmaf(l, r[i * step + 32], b);
    }
  }
  return make_float2(a, b);
}

// Rows X at the solution points interpolated to the flux points.
template <class C>
__global__ void __launch_bounds__(kThreads) k_fr_interp(const __grid_constant__ DevFormat F,
                                                        const __grid_constant__ FrBasisDev B,
                                                        FrSmem L, const typename C::T *X,
                                                        int64_t ne, int64_t ld, int nv,
                                                        typename C::T *Xf) {
  extern __shared__ __align__(16) unsigned char smem[];
  C codec = CodecOf<C>::make(F, smem, L);
  float *sx = reinterpret_cast<float *>(smem + L.off_stage);  // [ns][3][64]
  const int q = B.q, ns = q * q * q, nf = 6 * q * q;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t ntiles = (ne + kTile - 1) / kTile;
  const int64_t items = ntiles * nv;
  const int64_t cs_in = (int64_t)ns * nv * ld, cs_out = (int64_t)nf * nv * ld;
  for (int64_t it = blockIdx.x; it < items; it += gridDim.x) {
    const int64_t e0 = (it / nv) * kTile;
    const int v = (int)(it % nv);
    const int64_t ea = e0 + lane, eb = e0 + lane + 32;
    const bool va = ea < ne, vb = eb < ne;
    stage_rows<C::kWords>(codec, X, sx, ns, nv, v, ld, e0, ne, cs_in);
    __syncthreads();
    for (int f = warp; f < nf; f += kWarps) {
      const FaceLine fl = face_line(B, f);
      const float2 x = line_value(sx, B, fl, 0, lane);
      const float2 y = line_value(sx, B, fl, 1, lane);
      const float2 z = line_value(sx, B, fl, 2, lane);
      const int64_t idx = ((int64_t)f * nv + v) * ld;
      codec.store2(Xf, idx + ea, idx + eb, va, vb, cs_out, x, y, z);
    }
    __syncthreads();
  }
  codec.finish();
}

// F^fc = nF - sign(side) e_c . (F interpolated to the flux point).
template <class C>
__global__ void __launch_bounds__(kThreads) k_fr_fcorr(const __grid_constant__ DevFormat F,
                                                       const __grid_constant__ FrBasisDev B,
                                                       FrSmem L, const typename C::T *Fs,
                                                       const float *__restrict__ nF,
                                                       int64_t ne, int64_t ld, int nv,
                                                       float *Fc) {
  extern __shared__ __align__(16) unsigned char smem[];
  C codec = CodecOf<C>::make(F, smem, L);
  float *sx = reinterpret_cast<float *>(smem + L.off_stage);
  const int q = B.q, ns = q * q * q, nf = 6 * q * q;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t ntiles = (ne + kTile - 1) / kTile;
  const int64_t items = ntiles * nv;
  const int64_t cs_in = (int64_t)ns * nv * ld;
  for (int64_t it = blockIdx.x; it < items; it += gridDim.x) {
    const int64_t e0 = (it / nv) * kTile;
    const int v = (int)(it % nv);
    const int64_t ea = e0 + lane, eb = e0 + lane + 32;
    const bool va = ea < ne, vb = eb < ne;
    // the interface fluxes are loaded one point ahead, the first before the
    // staging, so that their latency overlaps the work
    auto nf_at = [&](int f) {
      float2 r = make_float2(0.0f, 0.0f);
      if (f < nf) {
        const int64_t idx = ((int64_t)f * nv + v) * ld;
        if (va) r.x = __ldg(nF + idx + ea);
        if (vb) r.y = __ldg(nF + idx + eb);
      }
      return r;
    };
    float2 nfc = nf_at(warp);
    stage_rows<false>(codec, Fs, sx, ns, nv, v, ld, e0, ne, cs_in);
    __syncthreads();
    for (int f = warp; f < nf; f += kWarps) {
      const float2 nfn = nf_at(f + kWarps);
      const FaceLine fl = face_line(B, f);
      const float2 t = line_value(sx, B, fl, fl.axis, lane);
      const float sg = fl.side ? 1.0f : -1.0f;
      const int64_t idx = ((int64_t)f * nv + v) * ld;
      if (va) Fc[idx + ea] = fmaf(-sg, t.x, nfc.x);
      if (vb) Fc[idx + eb] = fmaf(-sg, t.y, nfc.y);
      nfc = nfn;
    }
    __syncthreads();
  }
  codec.finish();
}

// ------------------------------------------------------------ physics (8, 9)

// Physical gradients of the primitives: (S^T G) / |J|.
__device__ __forceinline__ void physical_gradient(const float G[5][3], const float S[3][3],
                                                  float detJ, float gx[5][3]) {
  const float r = 1.0f / detJ;
  for (int v = 0; v < 5; ++v)
    for (int i = 0; i < 3; ++i)
      gx[v][i] = fmaf(S[2][i], G[v][2], fmaf(S[1][i], G[v][1], S[0][i] * G[v][0])) * r;
}

// Viscous flux rows 1..4 (row 0 is zero) of conserved q with physical
// primitive gradients gx: the stress (Stokes hypothesis) and u . tau +
// kappa grad(p / rho).
__device__ __forceinline__ void viscous_rows(const float qv[5], const float gx[5][3],
                                             const FrGasDev &gas, float Fv[4][3]) {
  const float rinv = 1.0f / qv[0];
  const float u[3] = {qv[1] * rinv, qv[2] * rinv, qv[3] * rinv};
  const float ke = 0.5f * qv[0] * fmaf(u[2], u[2], fmaf(u[1], u[1], u[0] * u[0]));
  const float p = (gas.gamma - 1.0f) * (qv[4] - ke);
  const float div = gx[1][0] + gx[2][1] + gx[3][2];
  const float t = p * rinv;
  for (int b = 0; b < 3; ++b)
    for (int a = 0; a < 3; ++a) {
      float tau = gas.mu * (gx[1 + b][a] + gx[1 + a][b]);
      if (a == b) tau = fmaf(-(2.0f / 3.0f) * gas.mu, div, tau);
      Fv[b][a] = tau;
    }
  for (int a = 0; a < 3; ++a) {
    const float gradt = fmaf(-t, gx[0][a], gx[4][a]) * rinv;
    Fv[3][a] = fmaf(gas.kappa, gradt,
                    fmaf(u[2], Fv[2][a], fmaf(u[1], Fv[1][a], u[0] * Fv[0][a])));
  }
}

// Reference flux rows S (F_inv - F_vis) at one point.
__device__ __forceinline__ void point_flux(const float qv[5], const float G[5][3],
                                           const float S[3][3], float detJ,
                                           const FrGasDev &gas, float out[5][3]) {
  float gx[5][3];
  physical_gradient(G, S, detJ, gx);
  float Fv[4][3];
  viscous_rows(qv, gx, gas, Fv);
  const float rinv = 1.0f / qv[0];
  const float u[3] = {qv[1] * rinv, qv[2] * rinv, qv[3] * rinv};
  const float ke = 0.5f * qv[0] * fmaf(u[2], u[2], fmaf(u[1], u[1], u[0] * u[0]));
  const float p = (gas.gamma - 1.0f) * (qv[4] - ke);
  float Fp[5][3];
  for (int a = 0; a < 3; ++a) {
    Fp[0][a] = qv[1 + a];
    for (int i = 0; i < 3; ++i) Fp[1 + i][a] = fmaf(qv[1 + i], u[a], i == a ? p : 0.0f) - Fv[i][a];
    Fp[4][a] = fmaf(qv[4] + p, u[a], -Fv[3][a]);
  }
  for (int v = 0; v < 5; ++v)
    for (int r = 0; r < 3; ++r)
      out[v][r] = fmaf(S[r][2], Fp[v][2], fmaf(S[r][1], Fp[v][1], S[r][0] * Fp[v][0]));
}

// The inputs of the pointwise physics at one point for two elements: every
// load of the point is issued before the first decode, so the decodes wait
// for memory once.
template <class C>
struct PointIn {
  float qa[5], qb[5], ja, jb;
  typename C::Raw g[5], s[3];

  __device__ void fetch(const C &codec, const float *qsrc, const typename C::T *G,
                        const typename C::T *S, const float *detJ, int k, int64_t ea, int64_t eb,
                        bool va, bool vb, int64_t ld, int64_t cs5, int64_t cs3) {
    for (int v = 0; v < 5; ++v) {
      const int64_t idx = ((int64_t)k * 5 + v) * ld;
      qa[v] = va ? __ldg(qsrc + idx + ea) : 1.0f;
      qb[v] = vb ? __ldg(qsrc + idx + eb) : 1.0f;
      g[v] = codec.fetch2(G, idx + ea, idx + eb, va, vb, cs5);
    }
    for (int r = 0; r < 3; ++r) {
      const int64_t idx = ((int64_t)k * 3 + r) * ld;
      s[r] = codec.fetch2(S, idx + ea, idx + eb, va, vb, cs3);
    }
    ja = va ? __ldg(detJ + (int64_t)k * ld + ea) : 1.0f;
    jb = vb ? __ldg(detJ + (int64_t)k * ld + eb) : 1.0f;
  }
};

// Splits a pair of rows into per-element arrays.
__device__ __forceinline__ void unpair(float2 X, float2 Y, float2 Z, float a[3], float b[3]) {
  a[0] = X.x; a[1] = Y.x; a[2] = Z.x;
  b[0] = X.y; b[1] = Y.y; b[2] = Z.y;
}

// Step 9: F^s rows from q^s, grad w^s rows, metric rows S and |J| (FP32 rows;
// compressed rows run k_fr_flux_w).
template <class C>
__global__ void __launch_bounds__(kThreads) k_fr_flux(const __grid_constant__ DevFormat F,
                                                      FrGasDev gas, FrSmem L, int ns,
                                                      const float *__restrict__ qs,
                                                      const typename C::T *G,
                                                      const typename C::T *S,
                                                      const float *__restrict__ detJ,
                                                      int64_t ne, int64_t ld,
                                                      typename C::T *Fs) {
  extern __shared__ __align__(16) unsigned char smem[];
  C codec = CodecOf<C>::make(F, smem, L);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t ntiles = (ne + kTile - 1) / kTile;
  const int64_t cs5 = (int64_t)ns * 5 * ld, cs3 = (int64_t)ns * 3 * ld;
  const int64_t gw = (int64_t)blockIdx.x * kWarps + warp, nw = (int64_t)gridDim.x * kWarps;
  for (ItemWalk iw(gw, nw, ns); iw.tile < ntiles; iw.next()) {
    const int64_t e0 = iw.tile * kTile;
    const int k = iw.sub;
    const int64_t ea = e0 + lane, eb = e0 + lane + 32;
    const bool va = ea < ne, vb = eb < ne;
    PointIn<C> in;
    in.fetch(codec, qs, G, S, detJ, k, ea, eb, va, vb, ld, cs5, cs3);
    float Ga[5][3], Gb[5][3], Sa[3][3], Sb[3][3];
    for (int v = 0; v < 5; ++v) {
      float2 X, Y, Z;
      codec.decode_raw(in.g[v], X, Y, Z);
      unpair(X, Y, Z, Ga[v], Gb[v]);
    }
    for (int r = 0; r < 3; ++r) {
      float2 X, Y, Z;
      codec.decode_raw(in.s[r], X, Y, Z);
      unpair(X, Y, Z, Sa[r], Sb[r]);
    }
    float Fa[5][3], Fb[5][3];
    point_flux(in.qa, Ga, Sa, in.ja, gas, Fa);
    point_flux(in.qb, Gb, Sb, in.jb, gas, Fb);
    for (int v = 0; v < 5; ++v) {
      const int64_t idx = ((int64_t)k * 5 + v) * ld;
      codec.store2(Fs, idx + ea, idx + eb, va, vb, cs5, make_float2(Fa[v][0], Fb[v][0]),
                   make_float2(Fa[v][1], Fb[v][1]), make_float2(Fa[v][2], Fb[v][2]));
    }
  }
  codec.finish();
}

// The element across face (c, s) of element e on a periodic Ex x Ey x Ez
// mesh, e = (ez Ey + ey) Ex + ex.  Two 32-bit divisions where the mesh has
// fewer than 2^32 elements (always, in practice), 64-bit ones otherwise.
__device__ __forceinline__ int64_t neighbour(int64_t e, int c, int s, int Ex, int Ey, int Ez) {
  int64_t ix, iy, iz;
  const int64_t exy = (int64_t)Ex * Ey;
  if (exy * Ez <= (int64_t)0xffffffffu) {
    const uint32_t u = (uint32_t)e, uxy = (uint32_t)exy;
    const uint32_t z = u / uxy, r = u - z * uxy, y = r / (uint32_t)Ex;
    ix = r - y * (uint32_t)Ex;
    iy = y;
    iz = z;
  } else {
    ix = e % Ex;
    iy = (e / Ex) % Ey;
    iz = e / exy;
  }
  const int d = s ? 1 : -1;
  if (c == 0) ix = ix + d == Ex ? 0 : (ix + d < 0 ? Ex - 1 : ix + d);
  else if (c == 1) iy = iy + d == Ey ? 0 : (iy + d < 0 ? Ey - 1 : iy + d);
  else iz = iz + d == Ez ? 0 : (iz + d < 0 ? Ez - 1 : iz + d);
  return (iz * Ey + iy) * Ex + ix;
}

// Viscous flux rows of one side from its fetched inputs (FP32 rows).
template <class C>
__device__ __forceinline__ void side_viscous_from(const C &codec, const PointIn<C> &in,
                                                  const FrGasDev &gas, float Fa[4][3],
                                                  float Fb[4][3]) {
  float Ga[5][3], Gb[5][3], Sa[3][3], Sb[3][3];
  for (int v = 0; v < 5; ++v) {
    float2 X, Y, Z;
    codec.decode_raw(in.g[v], X, Y, Z);
    unpair(X, Y, Z, Ga[v], Gb[v]);
  }
  for (int r = 0; r < 3; ++r) {
    float2 X, Y, Z;
    codec.decode_raw(in.s[r], X, Y, Z);
    unpair(X, Y, Z, Sa[r], Sb[r]);
  }
  float gx[5][3];
  physical_gradient(Ga, Sa, in.ja, gx);
  viscous_rows(in.qa, gx, gas, Fa);
  physical_gradient(Gb, Sb, in.jb, gx);
  viscous_rows(in.qb, gx, gas, Fb);
}

// Step 8: n . (F_inv - F^I_vis) at every flux point of every element, with
// F^I_vis the mean of the two sides' viscous fluxes (BR1).  Each interface is
// evaluated once: the thread of flux point f on the + face of axis c of
// element e also writes the matching point f - q^2 on the - face of the
// neighbour e' across it (a bijection on a periodic mesh, so every output has
// one writer), and each side's rows are read once.  FP32 rows; compressed
// rows run k_fr_commonvis_w.
template <class C>
__global__ void __launch_bounds__(kThreads, 1) k_fr_commonvis(
    const __grid_constant__ DevFormat F, FrGasDev gas, FrSmem L, int q, int Ex, int Ey, int Ez,
    const typename C::T *G, const typename C::T *nrm, const typename C::T *S,
    const float *__restrict__ detJ, const float *__restrict__ qf, const float *__restrict__ nFinv,
    int64_t ne, int64_t ld, float *out) {
  extern __shared__ __align__(16) unsigned char smem[];
  C codec = CodecOf<C>::make(F, smem, L);
  const int nf = 6 * q * q, nplus = 3 * q * q;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t ntiles = (ne + kTile - 1) / kTile;
  const int64_t cs5 = (int64_t)nf * 5 * ld, cs3 = (int64_t)nf * 3 * ld, cs1 = (int64_t)nf * ld;
  const int64_t gw = (int64_t)blockIdx.x * kWarps + warp, nw = (int64_t)gridDim.x * kWarps;
  const int qq = q * q;
  for (ItemWalk iw(gw, nw, nplus); iw.tile < ntiles; iw.next()) {
    const int64_t e0 = iw.tile * kTile;
    const int j = iw.sub;                           // + face point: axis c, in-face index
    const int c = (j >= qq) + (j >= 2 * qq);
    const int f = (2 * c + 1) * qq + (j - c * qq), fo = f - qq;
    const int64_t ea = e0 + lane, eb = e0 + lane + 32;
    const bool va = ea < ne, vb = eb < ne;
    const int64_t pa = va ? neighbour(ea, c, 1, Ex, Ey, Ez) : 0;
    const int64_t pb = vb ? neighbour(eb, c, 1, Ex, Ey, Ez) : 0;
    float Fa[4][3], Fb[4][3], Pa[4][3], Pb[4][3];
    PointIn<C> in0, in1;                            // both sides' loads in flight at once
    in0.fetch(codec, qf, G, S, detJ, f, ea, eb, va, vb, ld, cs5, cs3);
    in1.fetch(codec, qf, G, S, detJ, fo, pa, pb, va, vb, ld, cs5, cs3);
    side_viscous_from(codec, in0, gas, Fa, Fb);
    side_viscous_from(codec, in1, gas, Pa, Pb);
    float2 nx, ny, nz, mx, my, mz;
    codec.load2(nrm, (int64_t)f * ld + ea, (int64_t)f * ld + eb, va, vb, cs1, nx, ny, nz);
    codec.load2(nrm, (int64_t)fo * ld + pa, (int64_t)fo * ld + pb, va, vb, cs1, mx, my, mz);
    for (int v = 0; v < 5; ++v) {
      const int64_t idx = ((int64_t)f * 5 + v) * ld, ido = ((int64_t)fo * 5 + v) * ld;
      if (v == 0) {
        if (va) {
          out[idx + ea] = __ldg(nFinv + idx + ea);
          out[ido + pa] = __ldg(nFinv + ido + pa);
        }
        if (vb) {
          out[idx + eb] = __ldg(nFinv + idx + eb);
          out[ido + pb] = __ldg(nFinv + ido + pb);
        }
        continue;
      }
      const float *fa = Fa[v - 1], *fb = Fb[v - 1], *ga = Pa[v - 1], *gb = Pb[v - 1];
      const float sa0 = fa[0] + ga[0], sa1 = fa[1] + ga[1], sa2 = fa[2] + ga[2];
      const float sb0 = fb[0] + gb[0], sb1 = fb[1] + gb[1], sb2 = fb[2] + gb[2];
      if (va) {
        out[idx + ea] = fmaf(-0.5f, fmaf(nz.x, sa2, fmaf(ny.x, sa1, nx.x * sa0)),
                             __ldg(nFinv + idx + ea));
        out[ido + pa] = fmaf(-0.5f, fmaf(mz.x, sa2, fmaf(my.x, sa1, mx.x * sa0)),
                             __ldg(nFinv + ido + pa));
      }
      if (vb) {
        out[idx + eb] = fmaf(-0.5f, fmaf(nz.y, sb2, fmaf(ny.y, sb1, nx.y * sb0)),
                             __ldg(nFinv + idx + eb));
        out[ido + pb] = fmaf(-0.5f, fmaf(mz.y, sb2, fmaf(my.y, sb1, mx.y * sb0)),
                             __ldg(nFinv + ido + pb));
      }
    }
  }
  codec.finish();
}

// ------------------------------------------------------------ word rows of steps 8, 9
//
// The pointwise steps read eight compressed rows per point and side (gradient
// rows 0-4, metric rows 5-7).  Their decode loop stays rolled (an inlined
// decoder per row made these kernels 2-3x slower), so the rows it reads and
// writes live in per-thread shared-memory slots instead of local memory:
// slot s of a thread is one pair of FP32 values (elements lane and lane + 32)
// at float2 index s * kThreads + threadIdx.x, conflict-free.  The raw words
// arrive by cp.async, holding no registers while in flight, in slots that no
// decode overwrites before reading them: raw row j at R + 2j, R + 2j + 1, its
// decoded row at D + 3j .. D + 3j + 2, with R - D >= 8 (then D + 3j + 2 <
// R + 2(j + 1) for every j < 8).  The FP32-row twins have no decode and keep
// their rows in registers (k_fr_flux, k_fr_commonvis).

constexpr int kRows = 8;

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// 8-byte asynchronous global-to-shared copy; bytes = 0 fills zeros without
// reading the source.
__device__ __forceinline__ void cp_async8(void *dst, const void *src, uint32_t bytes) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(smem_u32(dst)),
               "l"(__cvta_generic_to_global(src)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;" ::: "memory");
}

template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Starts the copies of point k's raw rows (elements ea, eb; an absent element
// reads as the zero word) into this thread's slots R + 2j, R + 2j + 1.
__device__ __forceinline__ void fetch_rows_async(float2 *sc, int R, const uint64_t *G,
                                                 const uint64_t *S, int k, int64_t ea,
                                                 int64_t eb, bool va, bool vb, int64_t ld) {
#pragma unroll
  for (int j = 0; j < kRows; ++j) {
    const uint64_t *row = j < 5 ? G + ((int64_t)k * 5 + j) * ld : S + ((int64_t)k * 3 + j - 5) * ld;
    cp_async8(sc + (R + 2 * j) * kThreads, va ? row + ea : row, va ? 8u : 0u);
    cp_async8(sc + (R + 2 * j + 1) * kThreads, vb ? row + eb : row, vb ? 8u : 0u);
  }
}

// The word held in a slot (read as the slot's own type).
__device__ __forceinline__ uint64_t slot_word(const float2 *p) {
  const float2 t = *p;
  return ((uint64_t)__float_as_uint(t.y) << 32) | __float_as_uint(t.x);
}

// Decodes the eight raw rows at R into pairs at D (one decoder in the code).
template <class C>
__device__ __forceinline__ void decode_rows(const C &codec, float2 *sc, int R, int D) {
#pragma unroll 1
  for (int j = 0; j < kRows; ++j) {
    typename C::Raw r;
    r.w0 = slot_word(sc + (R + 2 * j) * kThreads);
    r.w1 = slot_word(sc + (R + 2 * j + 1) * kThreads);
    float2 X, Y, Z;
    codec.decode_raw(r, X, Y, Z);
    sc[(D + 3 * j) * kThreads] = X;
    sc[(D + 3 * j + 1) * kThreads] = Y;
    sc[(D + 3 * j + 2) * kThreads] = Z;
  }
}

template <int H>
__device__ __forceinline__ float half_of(const float2 *p) {
  return H ? p->y : p->x;
}

template <int H>
__device__ __forceinline__ void set_half(float2 *p, float v) {
  if (H) p->y = v;
  else p->x = v;
}

// Gradient and metric rows of element half H from the decoded rows at D.
template <int H>
__device__ __forceinline__ void side_rows(const float2 *sc, int D, float G[5][3], float S[3][3]) {
#pragma unroll
  for (int v = 0; v < 5; ++v)
#pragma unroll
    for (int i = 0; i < 3; ++i) G[v][i] = half_of<H>(sc + (D + 3 * v + i) * kThreads);
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int i = 0; i < 3; ++i) S[r][i] = half_of<H>(sc + (D + 15 + 3 * r + i) * kThreads);
}

// Step 9 for element half H: its flux rows replace the decoded rows 0-4 at D
// (read in full before the first write).
template <int H>
__device__ __forceinline__ void half_flux(float2 *sc, int D, const float qv[5], float detJ,
                                          const FrGasDev &gas) {
  float G[5][3], S[3][3], Fo[5][3];
  side_rows<H>(sc, D, G, S);
  point_flux(qv, G, S, detJ, gas, Fo);
#pragma unroll
  for (int v = 0; v < 5; ++v)
#pragma unroll
    for (int i = 0; i < 3; ++i) set_half<H>(sc + (D + 3 * v + i) * kThreads, Fo[v][i]);
}

// Step 8 for element half H of one side: its viscous rows 1-4 replace the
// decoded slots D .. D + 11.
template <int H>
__device__ __forceinline__ void half_viscous(float2 *sc, int D, const float qv[5], float detJ,
                                             const FrGasDev &gas) {
  float G[5][3], S[3][3], gx[5][3], Fv[4][3];
  side_rows<H>(sc, D, G, S);
  physical_gradient(G, S, detJ, gx);
  viscous_rows(qv, gx, gas, Fv);
#pragma unroll
  for (int b = 0; b < 4; ++b)
#pragma unroll
    for (int a = 0; a < 3; ++a) set_half<H>(sc + (D + 3 * b + a) * kThreads, Fv[b][a]);
}

// Conserved variables and |J| of point k for both elements (1 when absent).
__device__ __forceinline__ void point_scalars(const float *qsrc, const float *detJ, int k,
                                              int64_t ea, int64_t eb, bool va, bool vb,
                                              int64_t ld, float qa[5], float qb[5], float &ja,
                                              float &jb) {
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    const int64_t idx = ((int64_t)k * 5 + v) * ld;
    qa[v] = va ? __ldg(qsrc + idx + ea) : 1.0f;
    qb[v] = vb ? __ldg(qsrc + idx + eb) : 1.0f;
  }
  ja = va ? __ldg(detJ + (int64_t)k * ld + ea) : 1.0f;
  jb = vb ? __ldg(detJ + (int64_t)k * ld + eb) : 1.0f;
}

constexpr int kFluxSlots = 24;       // step 9: decoded rows 0-23, raw rows 8-23
constexpr int kInterfaceSlots = 44;  // step 8: see k_fr_commonvis_w

// Step 9 on compressed rows (same results as k_fr_flux).
template <class C>
__global__ void __launch_bounds__(kThreads) k_fr_flux_w(const __grid_constant__ DevFormat F,
                                                        FrGasDev gas, FrSmem L, int ns,
                                                        const float *__restrict__ qs,
                                                        const uint64_t *G, const uint64_t *S,
                                                        const float *__restrict__ detJ,
                                                        int64_t ne, int64_t ld, uint64_t *Fs) {
  extern __shared__ __align__(16) unsigned char smem[];
  C codec = CodecOf<C>::make(F, smem, L);
  float2 *sc = reinterpret_cast<float2 *>(smem + L.off_stage) + threadIdx.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t ntiles = (ne + kTile - 1) / kTile;
  const int64_t gw = (int64_t)blockIdx.x * kWarps + warp, nw = (int64_t)gridDim.x * kWarps;
  for (ItemWalk iw(gw, nw, ns); iw.tile < ntiles; iw.next()) {
    const int64_t e0 = iw.tile * kTile;
    const int k = iw.sub;
    const int64_t ea = e0 + lane, eb = e0 + lane + 32;
    const bool va = ea < ne, vb = eb < ne;
    fetch_rows_async(sc, 8, G, S, k, ea, eb, va, vb, ld);
    cp_async_commit();
    float qa[5], qb[5], ja, jb;
    point_scalars(qs, detJ, k, ea, eb, va, vb, ld, qa, qb, ja, jb);
    cp_async_wait<0>();
    decode_rows(codec, sc, 8, 0);
    half_flux<0>(sc, 0, qa, ja, gas);
    half_flux<1>(sc, 0, qb, jb, gas);
#pragma unroll 1
    for (int v = 0; v < 5; ++v) {
      const int64_t idx = ((int64_t)k * 5 + v) * ld;
      codec.store2(Fs, idx + ea, idx + eb, va, vb, 0, sc[(3 * v) * kThreads],
                   sc[(3 * v + 1) * kThreads], sc[(3 * v + 2) * kThreads]);
    }
  }
  codec.finish();
}

// Step 8 on compressed rows (same results and pairing of the sides as
// k_fr_commonvis).  Slots: this side's rows decoded at 0-23 from raw 8-23, its
// viscous rows then at 0-11; the other side's raw rows at 24-39, copied while
// this side is decoded, decoded at 12-35, viscous rows at 12-23; the two
// normal rows raw at 40-43.
template <class C>
__global__ void __launch_bounds__(kThreads, 2) k_fr_commonvis_w(
    const __grid_constant__ DevFormat F, FrGasDev gas, FrSmem L, int q, int Ex, int Ey, int Ez,
    const uint64_t *G, const uint64_t *nrm, const uint64_t *S, const float *__restrict__ detJ,
    const float *__restrict__ qf, const float *__restrict__ nFinv, int64_t ne, int64_t ld,
    float *out) {
  extern __shared__ __align__(16) unsigned char smem[];
  C codec = CodecOf<C>::make(F, smem, L);
  float2 *sc = reinterpret_cast<float2 *>(smem + L.off_stage) + threadIdx.x;
  const int nplus = 3 * q * q;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t ntiles = (ne + kTile - 1) / kTile;
  const int64_t gw = (int64_t)blockIdx.x * kWarps + warp, nw = (int64_t)gridDim.x * kWarps;
  const int qq = q * q;
  for (ItemWalk iw(gw, nw, nplus); iw.tile < ntiles; iw.next()) {
    const int64_t e0 = iw.tile * kTile;
    const int j = iw.sub;                           // + face point: axis c, in-face index
    const int c = (j >= qq) + (j >= 2 * qq);
    const int f = (2 * c + 1) * qq + (j - c * qq), fo = f - qq;
    const int64_t ea = e0 + lane, eb = e0 + lane + 32;
    const bool va = ea < ne, vb = eb < ne;
    const int64_t pa = va ? neighbour(ea, c, 1, Ex, Ey, Ez) : 0;
    const int64_t pb = vb ? neighbour(eb, c, 1, Ex, Ey, Ez) : 0;
    const uint64_t *nf = nrm + (int64_t)f * ld, *no = nrm + (int64_t)fo * ld;
    fetch_rows_async(sc, 8, G, S, f, ea, eb, va, vb, ld);
    cp_async8(sc + 40 * kThreads, va ? nf + ea : nf, va ? 8u : 0u);
    cp_async8(sc + 41 * kThreads, vb ? nf + eb : nf, vb ? 8u : 0u);
    cp_async8(sc + 42 * kThreads, va ? no + pa : no, va ? 8u : 0u);
    cp_async8(sc + 43 * kThreads, vb ? no + pb : no, vb ? 8u : 0u);
    cp_async_commit();
    fetch_rows_async(sc, 24, G, S, fo, pa, pb, va, vb, ld);
    cp_async_commit();
    float qa[5], qb[5], ja, jb, pqa[5], pqb[5], pja, pjb;
    point_scalars(qf, detJ, f, ea, eb, va, vb, ld, qa, qb, ja, jb);
    point_scalars(qf, detJ, fo, pa, pb, va, vb, ld, pqa, pqb, pja, pjb);
    cp_async_wait<1>();
    decode_rows(codec, sc, 8, 0);
    half_viscous<0>(sc, 0, qa, ja, gas);
    half_viscous<1>(sc, 0, qb, jb, gas);
    cp_async_wait<0>();
    decode_rows(codec, sc, 24, 12);
    half_viscous<0>(sc, 12, pqa, pja, gas);
    half_viscous<1>(sc, 12, pqb, pjb, gas);
    float2 nx, ny, nz, mx, my, mz;
    codec.decode_raw(typename C::Raw{slot_word(sc + 40 * kThreads), slot_word(sc + 41 * kThreads)},
                     nx, ny, nz);
    codec.decode_raw(typename C::Raw{slot_word(sc + 42 * kThreads), slot_word(sc + 43 * kThreads)},
                     mx, my, mz);
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      const int64_t idx = ((int64_t)f * 5 + v) * ld, ido = ((int64_t)fo * 5 + v) * ld;
      if (v == 0) {
        if (va) {
          out[idx + ea] = __ldg(nFinv + idx + ea);
          out[ido + pa] = __ldg(nFinv + ido + pa);
        }
        if (vb) {
          out[idx + eb] = __ldg(nFinv + idx + eb);
          out[ido + pb] = __ldg(nFinv + ido + pb);
        }
        continue;
      }
      float2 s[3];
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const float2 u = sc[(3 * (v - 1) + a) * kThreads], w = sc[(12 + 3 * (v - 1) + a) * kThreads];
        s[a] = make_float2(u.x + w.x, u.y + w.y);
      }
      if (va) {
        out[idx + ea] = fmaf(-0.5f, fmaf(nz.x, s[2].x, fmaf(ny.x, s[1].x, nx.x * s[0].x)),
                             __ldg(nFinv + idx + ea));
        out[ido + pa] = fmaf(-0.5f, fmaf(mz.x, s[2].x, fmaf(my.x, s[1].x, mx.x * s[0].x)),
                             __ldg(nFinv + ido + pa));
      }
      if (vb) {
        out[idx + eb] = fmaf(-0.5f, fmaf(nz.y, s[2].y, fmaf(ny.y, s[1].y, nx.y * s[0].y)),
                             __ldg(nFinv + idx + eb));
        out[ido + pb] = fmaf(-0.5f, fmaf(mz.y, s[2].y, fmaf(my.y, s[1].y, mx.y * s[0].y)),
                             __ldg(nFinv + ido + pb));
      }
    }
  }
  codec.finish();
}

// ------------------------------------------------------------ launchers

int sm_count() {
  int dev = 0, n = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return 1;
  }
  return n > 0 ? n : 1;
}

template <typename K>
cudaError_t launch_shape(K kernel, size_t smem, int64_t blocks_needed, int *grid) {
  cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  int occ = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, kThreads, smem);
  if (e != cudaSuccess) return e;
  if (occ < 1) return cudaErrorInvalidConfiguration;
  int64_t g = (int64_t)sm_count() * occ;
  if (g > blocks_needed) g = blocks_needed;
  *grid = (int)(g < 1 ? 1 : g);
  return cudaSuccess;
}

size_t align16(size_t v) { return (v + 15) & ~(size_t)15; }

// Shared-memory plan of a codec and a staging buffer of `stage` bytes; the
// per-warp queues only for kernels that encode.
template <class C>
FrSmem smem_plan(const DevFormat &F, int map, size_t stage, size_t *total, bool encodes = true) {
  size_t tab = C::kWords ? align16(table_smem_bytes(F, map)) : 0;
  size_t queue = (C::kQueue && encodes)
                     ? (size_t)kWarps * fast::kQueueCap * sizeof(fast::PendItem) : 0;
  FrSmem L;
  L.off_queue = (int)tab;
  L.off_stage = (int)(tab + align16(queue));
  *total = L.off_stage + stage;
  return L;
}

FrBasisDev basis_dev(const ivc_fr_basis &b) {
  FrBasisDev B{};
  B.q = b.order + 1;
  for (int i = 0; i < B.q; ++i) {
    for (int a = 0; a < B.q; ++a) B.dm[i][a] = b.dm[i * B.q + a];
    B.lm[i] = b.lm[i];
    B.lp[i] = b.lp[i];
    B.gl[i] = b.gl[i];
    B.gr[i] = b.gr[i];
  }
  const int q = B.q;
  for (int f = 0; f < 6 * q * q; ++f) {
    int c, s, ijk[3];
    face_of(f, q, c, s, ijk);
    const int stride = c == 0 ? 1 : (c == 1 ? q : q * q);
    B.fdesc[f] = point_of(ijk, q) | (stride << 8) | (s << 16) | (c << 17);
  }
  for (int k = 0; k < q * q * q; ++k) {
    int ijk[3];
    point_ijk(k, q, ijk);
    int d = ijk[0] | (ijk[1] << 2) | (ijk[2] << 4);
    for (int c = 0; c < 3; ++c) d |= flux_point(c, 0, ijk, q) << (6 + 7 * c);
    B.pdesc[k] = d;
  }
  return B;
}

FrGasDev gas_dev(const ivc_fr_gas &g) {
  const double k = (double)g.mu * g.gamma / (((double)g.gamma - 1.0) * g.prandtl);
  return FrGasDev{g.gamma, g.mu, (float)k};
}

// Runs f with the codec for (map, F): the fast path where the layout has one,
// else the generic decoder and encoder; FP32 rows when f32.
template <class Fn>
cudaError_t with_codec(bool f32, int map, const DevFormat &F, Fn &&fn) {
  if (f32) return fn(F32Rows{});
  switch (fast::fast_geometry(map, F)) {
    case 1: return fn(FastRows<fast::GeoPrimary>{F, nullptr, nullptr, {}});
    default: break;
  }
  if (map == MAP_TANH) return fn(GenericRows<MAP_TANH>{F, nullptr, nullptr});
  if (map == MAP_FRACSPLIT) return fn(GenericRows<MAP_FRACSPLIT>{F, nullptr, nullptr});
  return fn(GenericRows<MAP_UNIFORM>{F, nullptr, nullptr});
}

}  // namespace

cudaError_t launch_fr(const FrCall &a, cudaStream_t st) {
  const FrBasisDev B = basis_dev(a.basis);
  const FrGasDev gas = gas_dev(a.gas);
  const int q = B.q, ns = q * q * q, nf = 6 * q * q;
  const int64_t ntiles = (a.ne + kTile - 1) / kTile;
  return with_codec(a.f32, a.map, a.F, [&](auto codec) -> cudaError_t {
    using C = decltype(codec);
    using T = typename C::T;
    size_t smem = 0;
    int grid = 1;
    cudaError_t e;
    switch (a.step) {
      case 5: {
        const FrSmem L = smem_plan<C>(a.F, a.map, (size_t)ns * kTile * 4, &smem);
        if ((e = launch_shape(k_fr_grad<C>, smem, ntiles * a.nv, &grid)) != cudaSuccess) return e;
        k_fr_grad<C><<<grid, kThreads, smem, st>>>(a.F, B, L, (const float *)a.in0, a.ne, a.ld,
                                                   a.nv, (T *)a.out);
        break;
      }
      case 6: {
        const FrSmem L = smem_plan<C>(a.F, a.map, (size_t)nf * kTile * 4, &smem);
        if ((e = launch_shape(k_fr_correct<C>, smem, ntiles * a.nv, &grid)) != cudaSuccess)
          return e;
        k_fr_correct<C><<<grid, kThreads, smem, st>>>(a.F, B, L, (const T *)a.in0,
                                                      (const float *)a.in1, a.ne, a.ld, a.nv,
                                                      (T *)a.out);
        break;
      }
      case 7: {
        const FrSmem L = smem_plan<C>(a.F, a.map, (size_t)ns * 3 * kTile * 4, &smem);
        if ((e = launch_shape(k_fr_interp<C>, smem, ntiles * a.nv, &grid)) != cudaSuccess)
          return e;
        k_fr_interp<C><<<grid, kThreads, smem, st>>>(a.F, B, L, (const T *)a.in0, a.ne, a.ld,
                                                     a.nv, (T *)a.out);
        break;
      }
      case 11: {
        const FrSmem L = smem_plan<C>(a.F, a.map, (size_t)ns * 3 * kTile * 4, &smem, false);
        if ((e = launch_shape(k_fr_fcorr<C>, smem, ntiles * a.nv, &grid)) != cudaSuccess)
          return e;
        k_fr_fcorr<C><<<grid, kThreads, smem, st>>>(a.F, B, L, (const T *)a.in0,
                                                    (const float *)a.in1, a.ne, a.ld, a.nv,
                                                    (float *)a.out);
        break;
      }
      case 9: {
        const int64_t warps = ntiles * ns;
        if constexpr (C::kWords) {
          const FrSmem L = smem_plan<C>(a.F, a.map, (size_t)kFluxSlots * kThreads * 8, &smem);
          if ((e = launch_shape(k_fr_flux_w<C>, smem, (warps + kWarps - 1) / kWarps, &grid)) !=
              cudaSuccess)
            return e;
          k_fr_flux_w<C><<<grid, kThreads, smem, st>>>(
              a.F, gas, L, ns, (const float *)a.in0, (const uint64_t *)a.in1,
              (const uint64_t *)a.in2, (const float *)a.in3, a.ne, a.ld, (uint64_t *)a.out);
        } else {
          const FrSmem L = smem_plan<C>(a.F, a.map, 0, &smem);
          if ((e = launch_shape(k_fr_flux<C>, smem, (warps + kWarps - 1) / kWarps, &grid)) !=
              cudaSuccess)
            return e;
          k_fr_flux<C><<<grid, kThreads, smem, st>>>(a.F, gas, L, ns, (const float *)a.in0,
                                                     (const T *)a.in1, (const T *)a.in2,
                                                     (const float *)a.in3, a.ne, a.ld,
                                                     (T *)a.out);
        }
        break;
      }
      case 8: {
        const int64_t warps = ntiles * (nf / 2);
        if constexpr (C::kWords) {
          const FrSmem L =
              smem_plan<C>(a.F, a.map, (size_t)kInterfaceSlots * kThreads * 8, &smem, false);
          if ((e = launch_shape(k_fr_commonvis_w<C>, smem, (warps + kWarps - 1) / kWarps,
                                &grid)) != cudaSuccess)
            return e;
          k_fr_commonvis_w<C><<<grid, kThreads, smem, st>>>(
              a.F, gas, L, q, a.dims[0], a.dims[1], a.dims[2], (const uint64_t *)a.in0,
              (const uint64_t *)a.in1, (const uint64_t *)a.in2, (const float *)a.in3,
              (const float *)a.in4, (const float *)a.in5, a.ne, a.ld, (float *)a.out);
        } else {
          const FrSmem L = smem_plan<C>(a.F, a.map, 0, &smem, false);
          if ((e = launch_shape(k_fr_commonvis<C>, smem, (warps + kWarps - 1) / kWarps,
                                &grid)) != cudaSuccess)
            return e;
          k_fr_commonvis<C><<<grid, kThreads, smem, st>>>(
              a.F, gas, L, q, a.dims[0], a.dims[1], a.dims[2], (const T *)a.in0,
              (const T *)a.in1, (const T *)a.in2, (const float *)a.in3, (const float *)a.in4,
              (const float *)a.in5, a.ne, a.ld, (float *)a.out);
        }
        break;
      }
      default:
        return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
  });
}

}  // namespace ivc
