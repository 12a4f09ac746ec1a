// Fast path for the paper's primary layout <0,7,22>-17-18, b7 = 80 (Sec. 3,
// Sec. 5), and for its fractional split at n_phi_max + 1 = floor(2^17.5)
// (Sec. 2.4), default range handling.  Same results as the generic
// path in ivc_device.cuh (shared tables, same error bounds, same exact
// integer fallbacks); organised for GB300 issue throughput:
//   * every thread carries two vectors and does their FP32 arithmetic with the
//     packed f32x2 instructions (__ffma2 / __fadd2 / __fmul2, sm_100+);
//   * field extraction, the exact angle folds and table addressing use float
//     arithmetic on exact small integers and magic-number rounding, keeping
//     the integer/compare pipe for the few decisions that need it;
//   * encoding estimates t with a float-float octant-reduced atan (error
//     below 0.0035 bin in t) and runs the error-free side-of-boundary test only
//     for coordinates within kEps of a rounding boundary, deferred to a
//     per-warp queue;
//   * vectors with |x|^2 outside [2^-64, 2^64) (zero, NaN, Inf, tiny, huge) and
//     non-finite words take the generic code, off the common path.
#pragma once
#include "ivc_device.cuh"

namespace ivc {
namespace fast {

constexpr float kMagic = 12582912.0f;   // 1.5 * 2^23
constexpr uint32_t kMagicBits = 0x4B400000u;
constexpr float kEps = 0.005f;      // bin-coordinate estimate error bound (with margin)
// the tanh map's estimate: the atan error scaled by the map's largest slope
// relative to the uniform map, gamma / tanh(gamma) <= 1.32 for gamma <= 1
constexpr float kEpsTanh = 0.0065f;
// Bin-coordinate shift between the direction of a vector v and that of
// RN(rho v) for a positive rho: each component moves by at most 2^-24
// relative (or, below the FP32 normal range, by an absolute amount far below
// 2^-24 |v| inside the fast window), which turns theta = atan2(y, x) and
// phi = atan2(|(x, y)|, z) by at most 2^-24 rad: n_max / (2 pi) 2^-24 or
// n_max / pi 2^-24 < 0.0025 bin, times at most 1.32 for the tanh map.
constexpr float kReuseEps = 0.004f;

// The layouts this path serves: grid sizes n_theta_max = N, n_phi_max = M,
// head-table steps 2^ST (theta grid pi m / N) and 2^SP (phi grid
// pi m / (2M)) with NT, NP entries, the magnitude field (exponent field of
// the high word, r^ from the high word, high word of an RN32 magnitude) and
// the packing of the angle codes (Fig. comp_regimes).
// <0,7,22>-17-18 (Sec. 3): E7 in bits 57..63 (E8 - 47), m22 in 35..56 (the
// top 22 of the 23 mantissa bits), n_phi in 18..34, n_theta in 0..17.
struct GeoPrimary {
  static constexpr int N = 262143, M = 131071;
  static constexpr int ST = 8, SP = 8, NT = 513, NP = 513;
  static constexpr int MAP = MAP_UNIFORM;
  // bin scales N / (2 pi) and M / pi as float-float head + tail
  static constexpr float CTH = 0x1.45f2b6p+15f, CTL = -0x1.404a5ep-10f;
  static constexpr float CPH = 0x1.45f264p+15f, CPL = -0x1.ce6e62p-13f;
  static constexpr uint32_t EALL = 127u;   // non-finite exponent field
  __device__ static uint32_t efield(uint32_t hi) { return hi >> 25; }
  __device__ static float mag(uint32_t hi) {
    return __uint_as_float(((hi >> 2) & 0xFFFFFFFEu) + (47u << 23));
  }
  __device__ static uint32_t hi_of(uint32_t rb) { return ((rb - (47u << 23)) << 2) & 0xFFFFFFF8u; }
  __device__ static void unpack(uint32_t hi, uint32_t lo, uint32_t &nt, uint32_t &np) {
    nt = lo & 0x3FFFFu;
    np = __funnelshift_r(lo, hi, 18) & 0x1FFFFu;
  }
  __device__ static uint64_t pack(uint32_t hi_mag, int np, int nt) {
    return ((uint64_t)(hi_mag | ((uint32_t)np >> 14)) << 32) |
           (((uint32_t)np << 18) | (uint32_t)nt);
  }
};

// Fractional split (Sec. 2.4) at n_phi_max + 1 = 185363, n_theta_max + 1 =
// floor(2^35 / 185363) = 185364: the magnitude as in <0,7,22>-17-18 and
// n_p = n_phi (N + 1) + n_theta in bits 0..34.
struct GeoSplit {
  static constexpr int N = 185363, M = 185362;
  static constexpr int ST = 7, SP = 8, NT = 725, NP = 725;
  static constexpr int MAP = MAP_FRACSPLIT;
  // bin scales N / (2 pi) and M / pi as float-float head + tail
  static constexpr float CTH = 0x1.ccf5cp+14f, CTL = 0x1.c5b442p-13f;
  static constexpr float CPH = 0x1.ccf51ep+15f, CPL = -0x1.8199ccp-10f;
  static constexpr uint32_t EALL = 127u;
  __device__ static uint32_t efield(uint32_t hi) { return hi >> 25; }
  __device__ static float mag(uint32_t hi) {
    return __uint_as_float(((hi >> 2) & 0xFFFFFFFEu) + (47u << 23));
  }
  __device__ static uint32_t hi_of(uint32_t rb) { return ((rb - (47u << 23)) << 2) & 0xFFFFFFF8u; }
  __device__ static void unpack(uint32_t hi, uint32_t lo, uint32_t &nt, uint32_t &np) {
    const uint64_t npk = ((uint64_t)(hi & 7u) << 32) | lo;
    const uint64_t q = npk / (uint64_t)(N + 1);
    nt = (uint32_t)(npk - q * (uint64_t)(N + 1));
    // codes beyond (M + 1)(N + 1) - 1 are not valid: n_phi clamped as in the
    // generic decoder
    np = q > (uint64_t)M ? (uint32_t)M : (uint32_t)q;
  }
  __device__ static uint64_t pack(uint32_t hi_mag, int np, int nt) {
    // n_p < 2^35: its bits 32..34 fill the three free low bits of hi_mag
    return ((uint64_t)hi_mag << 32) + ((uint64_t)np * (uint64_t)(N + 1) + (uint64_t)nt);
  }
};

// <0,7,23>-17-17 (Sec. 2.3): E7 in bits 57..63, m23 in 34..56, n_phi in
// 17..33, n_theta in 0..16.
struct GeoL1717 {
  static constexpr int N = 131071, M = 131071;
  static constexpr int ST = 7, SP = 8, NT = 513, NP = 513;
  static constexpr int MAP = MAP_UNIFORM;
  // bin scales N / (2 pi) and M / pi as float-float head + tail
  static constexpr float CTH = 0x1.45f264p+14f, CTL = -0x1.ce6e62p-14f;
  static constexpr float CPH = 0x1.45f264p+15f, CPL = -0x1.ce6e62p-13f;
  static constexpr uint32_t EALL = 127u;
  __device__ static uint32_t efield(uint32_t hi) { return hi >> 25; }
  __device__ static float mag(uint32_t hi) { return __uint_as_float((hi >> 2) + (47u << 23)); }
  __device__ static uint32_t hi_of(uint32_t rb) { return ((rb - (47u << 23)) << 2) & 0xFFFFFFFCu; }
  __device__ static void unpack(uint32_t hi, uint32_t lo, uint32_t &nt, uint32_t &np) {
    nt = lo & 0x1FFFFu;
    np = __funnelshift_r(lo, hi, 17) & 0x1FFFFu;
  }
  __device__ static uint64_t pack(uint32_t hi_mag, int np, int nt) {
    return ((uint64_t)(hi_mag | ((uint32_t)np >> 15)) << 32) |
           (((uint32_t)np << 17) | (uint32_t)nt);
  }
};

// <0,8,23>-16-17 (Sec. 2.3): the FP32 exponent and mantissa of RN32(r) in
// bits 33..63 (E8 in 56..63), n_phi in 17..32, n_theta in 0..16.
struct GeoL1617 {
  static constexpr int N = 131071, M = 65535;
  static constexpr int ST = 7, SP = 7, NT = 513, NP = 513;
  static constexpr int MAP = MAP_UNIFORM;
  // bin scales N / (2 pi) and M / pi as float-float head + tail
  static constexpr float CTH = 0x1.45f264p+14f, CTL = -0x1.ce6e62p-14f;
  static constexpr float CPH = 0x1.45f1cp+14f, CPL = 0x1.d32b58p-11f;
  static constexpr uint32_t EALL = 255u;
  __device__ static uint32_t efield(uint32_t hi) { return hi >> 24; }
  __device__ static float mag(uint32_t hi) { return __uint_as_float(hi >> 1); }
  __device__ static uint32_t hi_of(uint32_t rb) { return (rb << 1) & 0xFFFFFFFEu; }
  __device__ static void unpack(uint32_t hi, uint32_t lo, uint32_t &nt, uint32_t &np) {
    nt = lo & 0x1FFFFu;
    np = __funnelshift_r(lo, hi, 17) & 0xFFFFu;
  }
  __device__ static uint64_t pack(uint32_t hi_mag, int np, int nt) {
    return ((uint64_t)(hi_mag | ((uint32_t)np >> 15)) << 32) |
           (((uint32_t)np << 17) | (uint32_t)nt);
  }
};

// <0,7,22>-17-18 with the tanh companding map (Sec. 2.5) on both angles:
// the bit layout of GeoPrimary; the decoder reads cos/sin of every code's
// angle from per-code tables (global), the encoder interpolates the bin
// coordinate from node tables (shared memory) and decides against the
// per-boundary tables.  Format parameter gamma in (0, 1].
struct GeoTanh {
  static constexpr int N = 262143, M = 131071;
  static constexpr int ST = 8, SP = 8, NT = 0, NP = 0;
  static constexpr int MAP = MAP_TANH;
  static constexpr float CTH = 0.0f, CTL = 0.0f, CPH = 0.0f, CPL = 0.0f;  // unused
  static constexpr uint32_t EALL = 127u;
  __device__ static uint32_t efield(uint32_t hi) { return hi >> 25; }
  __device__ static float mag(uint32_t hi) {
    return __uint_as_float(((hi >> 2) & 0xFFFFFFFEu) + (47u << 23));
  }
  __device__ static uint32_t hi_of(uint32_t rb) { return ((rb - (47u << 23)) << 2) & 0xFFFFFFF8u; }
  __device__ static void unpack(uint32_t hi, uint32_t lo, uint32_t &nt, uint32_t &np) {
    nt = lo & 0x3FFFFu;
    np = __funnelshift_r(lo, hi, 18) & 0x1FFFFu;
  }
  __device__ static uint64_t pack(uint32_t hi_mag, int np, int nt) {
    return ((uint64_t)(hi_mag | ((uint32_t)np >> 14)) << 32) |
           (((uint32_t)np << 18) | (uint32_t)nt);
  }
};

// Field positions of each fast layout, checked against a format.
template <class G> struct GeoFields;
template <> struct GeoFields<GeoPrimary> {
  static constexpr uint32_t sh_phi = 18, sh_m = 35, sh_e = 57, mask_e = 127, mask_m = 0x3FFFFF;
  static constexpr int e_off = -47;
};
template <> struct GeoFields<GeoSplit> {
  static constexpr uint32_t sh_phi = 18, sh_m = 35, sh_e = 57, mask_e = 127, mask_m = 0x3FFFFF;
  static constexpr int e_off = -47;
};
template <> struct GeoFields<GeoL1717> {
  static constexpr uint32_t sh_phi = 17, sh_m = 34, sh_e = 57, mask_e = 127, mask_m = 0x7FFFFF;
  static constexpr int e_off = -47;
};
template <> struct GeoFields<GeoL1617> {
  static constexpr uint32_t sh_phi = 17, sh_m = 33, sh_e = 56, mask_e = 255, mask_m = 0x7FFFFF;
  static constexpr int e_off = 0;
};
template <> struct GeoFields<GeoTanh> {
  static constexpr uint32_t sh_phi = 18, sh_m = 35, sh_e = 57, mask_e = 127, mask_m = 0x3FFFFF;
  static constexpr int e_off = -47;
};

template <class G>
__host__ __device__ inline bool is_geo(const DevFormat &F) {
  using P = GeoFields<G>;
  return F.sh_phi == P::sh_phi && F.sh_m == P::sh_m && F.sh_e == P::sh_e &&
         F.mask_e == P::mask_e && F.mask_m == P::mask_m && F.e_off == P::e_off &&
         F.N == G::N && F.M == G::M && F.st == G::ST && F.sp == G::SP &&
         F.nent_t == G::NT && F.nent_p == G::NP && F.under_mode == 0 && F.over_mode == 0;
}

// Which fast layout a format is: 1 primary, 2 fractional split, 3
// <0,7,23>-17-17, 4 <0,8,23>-16-17, 5 the primary layout with the tanh map,
// 0 none.
__host__ __device__ inline int fast_geometry(int map, const DevFormat &F) {
  if (map == MAP_UNIFORM && is_geo<GeoPrimary>(F)) return 1;
  if (map == MAP_FRACSPLIT && is_geo<GeoSplit>(F)) return 2;
  if (map == MAP_UNIFORM && is_geo<GeoL1717>(F)) return 3;
  if (map == MAP_UNIFORM && is_geo<GeoL1617>(F)) return 4;
  if (map == MAP_TANH && is_geo<GeoTanh>(F) && F.gam > 0.0f && F.gam <= 1.0f) return 5;
  return 0;
}

__device__ __forceinline__ float2 bc(float v) { return make_float2(v, v); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, bc(-1.0f), a); }
__device__ __forceinline__ float2 sel2(bool c0, bool c1, float2 a, float2 b) {
  return make_float2(c0 ? a.x : b.x, c1 ? a.y : b.y);
}

struct FF2 {
  float2 h, l;
};

// ------------------------------------------------------------ trig (packed)

// Folded angle in [0, pi/4] as pi b / (2D) for both elements, with the role
// flags of the original angle.
struct Fold2 {
  float2 b;
  bool swap0, swap1, cneg0, cneg1;
};

// cos/sin magnitudes of pi b / (2D) for both elements from the shared table
// (entries at b = h 2^S).
template <int S>
__device__ __forceinline__ void sincos2(float2 b, const TabEntry *__restrict__ tab, float Kh,
                                        float Kl, FF2 &c, FF2 &s) {
  // h = nearest integer to b / 2^S (magic-number rounding), l = b - 2^S h
  const float2 hb = fma2(b, bc(1.0f / (float)(1 << S)), bc(kMagic));
  const float2 hf = add2(hb, bc(-kMagic));
  const float2 lf = fma2(hf, bc(-(float)(1 << S)), b);
  const uint32_t i0 = __float_as_uint(hb.x) - kMagicBits;
  const uint32_t i1 = __float_as_uint(hb.y) - kMagicBits;
  const TabEntry e0 = tab[i0];
  const TabEntry e1 = tab[i1];
  const float2 X = make_float2(e0.ch, e1.ch), Xl = make_float2(e0.cl, e1.cl);
  const float2 Y = make_float2(e0.sh, e1.sh), Yl = make_float2(e0.sl, e1.sl);
  const float2 bh = mul2(lf, bc(Kh));
  const float2 bl = add2(fma2(lf, bc(Kh), neg2(bh)), mul2(lf, bc(Kl)));
  // 1 - cos(beta) ~ beta^2 / 2 and sin(beta) - bh ~ bl - beta^3 / 6: every fast
  // layout has |beta| <= 128 pi / (2 * 262142) = 7.7e-4 (the same bound for the
  // 2^7-step grids of half the size), so the next terms, beta^4 / 24 < 2^-45.9
  // and beta^5 / 120 < 2^-48 relative to sin(beta), stay far below the 2^-40
  // decode ambiguity threshold
  const float2 b2 = mul2(bh, bh);
  const float2 u = mul2(b2, bc(0.5f));
  const float2 st = fma2(mul2(bh, b2), bc(-1.0f / 6.0f), bl);
  // cos(A + beta) = cA - cA u - sA sin(beta)
  const float2 P = mul2(Y, bh);
  const float2 Pe = fma2(Y, bh, neg2(P));
  const float2 Ch = sub2(X, P);
  const float2 Ce = sub2(sub2(X, Ch), P);
  float2 Cl = add2(Ce, Xl);
  Cl = sub2(Cl, Pe);
  Cl = fma2(neg2(X), u, Cl);
  Cl = fma2(neg2(Y), st, Cl);
  Cl = fma2(neg2(Yl), bh, Cl);
  // sin(A + beta) = sA - sA u + cA sin(beta)
  const float2 Q = mul2(X, bh);
  const float2 Qe = fma2(X, bh, neg2(Q));
  const float2 Sh = add2(Y, Q);
  const float2 Se = sub2(Q, sub2(Sh, Y));
  float2 Sl = add2(Se, Qe);
  Sl = add2(Sl, Yl);
  Sl = fma2(neg2(Y), u, Sl);
  Sl = fma2(X, st, Sl);
  Sl = fma2(Xl, bh, Sl);
  c.h = Ch; c.l = Cl;
  s.h = Sh; s.l = Sl;
}

// Exact fold of pi m / D, given |m| as exact float a in [0, D].
__device__ __forceinline__ Fold2 fold2(float2 a, float D) {
  Fold2 f;
  const float2 na = fma2(a, bc(-1.0f), bc(D));        // D - a
  f.cneg0 = a.x > na.x;
  f.cneg1 = a.y > na.y;
  const float2 a1 = make_float2(fminf(a.x, na.x), fminf(a.y, na.y));
  const float2 t2 = add2(a1, a1);
  const float2 nt2 = fma2(a1, bc(-2.0f), bc(D));      // D - 2 a1
  f.swap0 = t2.x > nt2.x;
  f.swap1 = t2.y > nt2.y;
  f.b = make_float2(fminf(t2.x, nt2.x), fminf(t2.y, nt2.y));
  return f;
}

// ----------------------------------------------------------------- decode

// Round-up (away from zero for magnitudes) of (Ph + Pl) with the ambiguity
// test of the generic path, for both elements.
__device__ __forceinline__ float2 ru_pair(float2 P, float2 T, bool &amb0, bool &amb1) {
  const float2 d = mul2(P, bc(kDecodeAmbig));
  const float2 x0 = __fadd2_ru(P, sub2(T, d));
  const float2 x1 = __fadd2_ru(P, add2(T, d));
  amb0 |= (x0.x != x1.x);
  amb1 |= (x0.y != x1.y);
  return x1;
}

// RU(r (a.h + a.l)) with a float-float a: returns (P, T) with P + T the value.
__device__ __forceinline__ void prod2(float2 r, FF2 a, float2 &P, float2 &T) {
  P = mul2(r, a.h);
  const float2 Pe = fma2(r, a.h, neg2(P));
  T = fma2(r, a.l, Pe);
}

__device__ __forceinline__ void prod3(FF2 R, FF2 a, float2 &P, float2 &T) {
  P = mul2(R.h, a.h);
  const float2 Pe = fma2(R.h, a.h, neg2(P));
  T = fma2(R.h, a.l, fma2(R.l, a.h, Pe));
}

__device__ __forceinline__ float apply_neg(float v, bool n) { return (n && v != 0.0f) ? -v : v; }

// Magnitude of a signed float-float pair (the tail keeps its sign relative to
// the head) and the head's sign as +-1.
__device__ __forceinline__ FF2 abs_ff2(float2 h, float2 l, float2 &sg) {
  sg = make_float2(copysignf(1.0f, h.x), copysignf(1.0f, h.y));
  FF2 m;
  m.h = mul2(h, sg);
  m.l = mul2(l, sg);
  return m;
}

// cos and sin (float-float magnitudes) of phi^ = pi n / M for both elements,
// and whether cos phi^ is negative.  PT: one 16-byte load per element from
// the per-code table of k = min(n, M - n) (cos(pi - a) = -cos a, sin(pi -
// a) = sin a), read through L2; otherwise the angle is folded onto [0, pi/4]
// and evaluated from the shared-memory head table and a Taylor step.
template <class G, bool PT>
__device__ __forceinline__ void phi_pair(uint32_t np0, uint32_t np1, const DevFormat &F,
                                         const TabEntry *__restrict__ tab_p, FF2 &cp, FF2 &sp,
                                         bool &cneg0, bool &cneg1) {
  if (PT) {
    const int m0 = G::M - (int)np0, m1 = G::M - (int)np1;
    cneg0 = (int)np0 > m0;
    cneg1 = (int)np1 > m1;
    const float4 *t = reinterpret_cast<const float4 *>(F.phi_tab);
    const float4 e0 = __ldg(t + min((int)np0, m0));
    const float4 e1 = __ldg(t + min((int)np1, m1));
    cp.h = make_float2(e0.x, e1.x);
    cp.l = make_float2(e0.y, e1.y);
    sp.h = make_float2(e0.z, e1.z);
    sp.l = make_float2(e0.w, e1.w);
  } else {
    const float2 npf = add2(make_float2(__uint_as_float(np0 | 0x4B000000u),
                                        __uint_as_float(np1 | 0x4B000000u)),
                            bc(-8388608.0f));
    // phi^ = pi (2 n_phi) / (2M)
    const Fold2 fp = fold2(add2(npf, npf), (float)(2 * G::M));
    FF2 cc, ss;
    sincos2<G::SP>(fp.b, tab_p, F.Kp_h, F.Kp_l, cc, ss);
    cp.h = sel2(fp.swap0, fp.swap1, ss.h, cc.h);
    cp.l = sel2(fp.swap0, fp.swap1, ss.l, cc.l);
    sp.h = sel2(fp.swap0, fp.swap1, cc.h, ss.h);
    sp.l = sel2(fp.swap0, fp.swap1, cc.l, ss.l);
    cneg0 = fp.cneg0;
    cneg1 = fp.cneg1;
  }
}

// Decodes two words; returns false in *ok for an element that needs the
// generic path (non-finite word or an ambiguous rounding).
// The tanh map's per-code table entries of a word pair, staged in shared
// memory by stage_entries (slot stride ss float4): theta^ of w0, of w1, phi^
// of w0, of w1.
struct Staged {
  const float4 *p;
  int ss;
};

template <class G, bool PT>
__device__ __forceinline__ void decode2(uint64_t w0, uint64_t w1, const DevFormat &F,
                                        const TabEntry *__restrict__ tab_t,
                                        const TabEntry *__restrict__ tab_p, float2 &X,
                                        float2 &Y, float2 &Z, bool &slow0, bool &slow1,
                                        const Staged *stg = nullptr) {
  const uint32_t hi0 = (uint32_t)(w0 >> 32), lo0 = (uint32_t)w0;
  const uint32_t hi1 = (uint32_t)(w1 >> 32), lo1 = (uint32_t)w1;
  const uint32_t E0 = G::efield(hi0), E1 = G::efield(hi1);
  // r^ from the magnitude field (Sec. 2.3); exponent field 0 is the zero vector
  const float r0 = E0 == 0u ? 0.0f : G::mag(hi0);
  const float r1 = E1 == 0u ? 0.0f : G::mag(hi1);
  slow0 = (E0 == G::EALL);
  slow1 = (E1 == G::EALL);
  // n_theta, n_phi as exact floats (magic-number conversion, codes < 2^23)
  uint32_t nt0, np0, nt1, np1;
  G::unpack(hi0, lo0, nt0, np0);
  G::unpack(hi1, lo1, nt1, np1);
  FF2 ct, st, cp, sp;
  float2 sgx, sgy, sgz;  // signs of cos(theta^), sin(theta^), cos(phi^) as +-1
  if constexpr (G::MAP == MAP_TANH) {
    // signed float-float cos/sin of every code's angle, read through L2
    const float4 *dt = reinterpret_cast<const float4 *>(F.dec_t);
    const float4 *dp = reinterpret_cast<const float4 *>(F.dec_p);
    const float4 a0 = stg ? stg->p[0] : __ldg(dt + nt0);
    const float4 a1 = stg ? stg->p[stg->ss] : __ldg(dt + nt1);
    const float4 b0 = stg ? stg->p[2 * stg->ss] : __ldg(dp + np0);
    const float4 b1 = stg ? stg->p[3 * stg->ss] : __ldg(dp + np1);
    ct = abs_ff2(make_float2(a0.x, a1.x), make_float2(a0.y, a1.y), sgx);
    st = abs_ff2(make_float2(a0.z, a1.z), make_float2(a0.w, a1.w), sgy);
    cp = abs_ff2(make_float2(b0.x, b1.x), make_float2(b0.y, b1.y), sgz);
    sp.h = make_float2(b0.z, b1.z);  // sin(phi^) >= 0
    sp.l = make_float2(b0.w, b1.w);
  } else {
    // phi^ first: with the per-code table its loads are in flight while
    // theta^ is evaluated
    bool pneg0, pneg1;
    if (stg) {
      // the per-code phi^ entries, staged (slots 2 and 3)
      const float4 e0 = stg->p[2 * stg->ss], e1 = stg->p[3 * stg->ss];
      pneg0 = (int)np0 > G::M - (int)np0;
      pneg1 = (int)np1 > G::M - (int)np1;
      cp.h = make_float2(e0.x, e1.x);
      cp.l = make_float2(e0.y, e1.y);
      sp.h = make_float2(e0.z, e1.z);
      sp.l = make_float2(e0.w, e1.w);
    } else {
      phi_pair<G, PT>(np0, np1, F, tab_p, cp, sp, pneg0, pneg1);
    }
    const float2 ntf = add2(make_float2(__uint_as_float(nt0 | 0x4B000000u),
                                        __uint_as_float(nt1 | 0x4B000000u)),
                            bc(-8388608.0f));
    // theta^ = pi (2 n_theta - N) / N
    const float2 mt = fma2(ntf, bc(2.0f), bc(-(float)G::N));
    const Fold2 ft = fold2(make_float2(fabsf(mt.x), fabsf(mt.y)), (float)G::N);
    FF2 cc, ss;
    sincos2<G::ST>(ft.b, tab_t, F.Kt_h, F.Kt_l, cc, ss);
    ct.h = sel2(ft.swap0, ft.swap1, ss.h, cc.h);
    ct.l = sel2(ft.swap0, ft.swap1, ss.l, cc.l);
    st.h = sel2(ft.swap0, ft.swap1, cc.h, ss.h);
    st.l = sel2(ft.swap0, ft.swap1, cc.l, ss.l);
    // cos(theta^) < 0 iff the fold reflected, sin(theta^) < 0 iff m < 0,
    // cos(phi^) < 0 iff n_phi > M / 2
    sgx = make_float2(ft.cneg0 ? -1.0f : 1.0f, ft.cneg1 ? -1.0f : 1.0f);
    sgy = make_float2(copysignf(1.0f, mt.x), copysignf(1.0f, mt.y));
    sgz = make_float2(pneg0 ? -1.0f : 1.0f, pneg1 ? -1.0f : 1.0f);
  }
  // x = r cos(theta) sin(phi), y = r sin(theta) sin(phi), z = r cos(phi)
  const float2 r = make_float2(r0, r1);
  FF2 R;
  prod2(r, sp, R.h, R.l);
  float2 P, T;
  bool a0 = false, a1 = false;
  prod3(R, ct, P, T);
  const float2 x = ru_pair(P, T, a0, a1);
  prod3(R, st, P, T);
  const float2 y = ru_pair(P, T, a0, a1);
  prod2(r, cp, P, T);
  const float2 z = ru_pair(P, T, a0, a1);
  slow0 |= a0;
  slow1 |= a1;
  // signs; (+0) added so that exact zeros are +0
  X = fma2(x, sgx, bc(0.0f));
  Y = fma2(y, sgy, bc(0.0f));
  Z = fma2(z, sgz, bc(0.0f));
}

// ----------------------------------------------------------------- encode

__device__ __forceinline__ float rcp_approx(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ float sqrt_approx(float x) {
  float r;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// beta = atan(mn / mx) in [0, pi/4] for 0 <= mn <= mx, as an unevaluated sum
// bh + bl with |error| < 5e-8 rad:
//   * q = mn / mx as a float-float qh + ql (approximate reciprocal, then the
//     exact residual mn - mx qh times it: the quotient's own error cancels);
//   * atan(q) = q + q^3 R(q^2), R a degree-7 polynomial from a
//     least-squares-minimax (Lawson) fit on [0, 1] (7.4e-9 in exact
//     arithmetic), kept as q + s so that FP32 rounding acts on s only;
//   * the ql term enters with the slope 1/(1 + q^2), taken as 1 - q^2/2
//     (ql is below half an ulp of q, so 12 % slope error is negligible).
// mx = 0 (zero vector in this plane) gives beta = 0.
__device__ __forceinline__ void atan_ratio2(float2 mn, float2 mx, float2 &bh, float2 &bl) {
  const float2 m = make_float2(fmaxf(mx.x, 1e-30f), fmaxf(mx.y, 1e-30f));
  const float2 r = make_float2(rcp_approx(m.x), rcp_approx(m.y));
  const float2 qh = mul2(mn, r);
  const float2 ql = mul2(fma2(neg2(m), qh, mn), r);
  const float2 q2 = mul2(qh, qh);
  float2 R = bc(0.002622244181111455f);
  R = fma2(R, q2, bc(-0.015132534317672253f));
  R = fma2(R, q2, bc(0.04112185537815094f));
  R = fma2(R, q2, bc(-0.07366705685853958f));
  R = fma2(R, q2, bc(0.10573931783437729f));
  R = fma2(R, q2, bc(-0.1418597549200058f));
  R = fma2(R, q2, bc(0.1999039649963379f));
  R = fma2(R, q2, bc(-0.33332985639572144f));
  const float2 sv = mul2(mul2(qh, q2), R);                 // q^3 R(q^2)
  bh = qh;
  bl = fma2(ql, fma2(q2, bc(-0.5f), bc(1.0f)), sv);
}

// Bin coordinate t = K0 + s1 * C * beta (K0 a multiple of 1/4, s1 = +-1,
// C = n_max / pi or n_max / (2 pi) in float-float), returned as floor and
// fraction computed without rounding the large sum: C beta = G + small with
// G = RN(Ch bh) and small = its exact rounding error (an FMA) plus the tail
// products, G = Gi + Gf with Gi integral, then t = [K0 + s1 Gi] + s1 (Gf +
// small).  Error below 0.002 bin.
struct BinCoord2 {
  float2 fl, fr;  // floor(t) (exact integer-valued floats) and t - floor(t)
};

__device__ __forceinline__ float2 floor2(float2 v) {  // |v| < 2^22
  return add2(__fadd2_rd(v, bc(kMagic)), bc(-kMagic));
}

__device__ __forceinline__ BinCoord2 bin_coord2(float2 K0, float2 s1, float2 bh, float2 bl, float Ch,
                                                float Cl) {
  const float2 G = mul2(bc(Ch), bh);                       // C beta, head
  // the head's exact rounding error and the tail products
  const float2 small = fma2(bc(Ch), bl, fma2(bc(Cl), bh, fma2(bc(Ch), bh, neg2(G))));
  const float2 Gi = floor2(G);
  const float2 gfrac = add2(sub2(G, Gi), small);          // in (-0.01, 1.01)
  const float2 hI = fma2(s1, Gi, K0);                     // exact, quarter-integral
  const float2 fi = floor2(hI);
  const float2 f = fma2(s1, gfrac, sub2(hI, fi));         // in (-1.02, 1.77)
  const float2 fl2 = floor2(f);
  BinCoord2 c;
  c.fl = add2(fi, fl2);
  c.fr = sub2(f, fl2);
  return c;
}

// pi, pi / 2 and pi / 1024 as float-float head + tail; 1024 / pi
constexpr float kPiH = 0x1.921fb6p+1f, kPiL = -0x1.777a5cp-24f;
constexpr float kPi2H = 0x1.921fb6p+0f, kPi2L = -0x1.777a5cp-25f;
constexpr float kNodeH = 0x1.921fb6p-9f, kNodeL = -0x1.777a5cp-34f;
constexpr float kNodeScale = 0x1.45f306p+8f;
constexpr int kTanhNodesT = 1025, kTanhNodesP = 513;  // nodes over [0, pi] and [0, pi/2]

// tanh map (Sec. 2.5): bin coordinate t(a) at the angle a = Ka + sa (bh +
// bl) (Ka in {0, pi/2, pi} in float-float, beta = bh + bl <= pi / 4 as
// atan_ratio2 returns it) from the
// nearest node j pi / 1024 of `tab` (nodes entries: floor t_j, t_j - floor
// t_j, t'_j, t''_j / 2) by the quadratic step t_j + t' d + t''/2 d^2, d =
// a - j pi / 1024 (|d| <= pi / 2048: the cubic term is below 1e-4 bin for
// gamma <= 1).  Returns floor t and t - floor t (within 1e-4 bin of the
// exact bin coordinate of a).
__device__ __forceinline__ BinCoord2 tanh_bin2(float2 Kah, float2 Kal, float2 sa, float2 bh,
                                               float2 bl, const TabEntry *__restrict__ tab,
                                               int nodes) {
  // beta = bh + bl with bl up to a fifth of bh (atan_ratio2's q and its
  // correction): renormalised to a head and a tail (Fast2Sum, |bh| >= |bl|)
  const float2 gh = add2(bh, bl);
  const float2 gl = add2(sub2(bh, gh), bl);
  // a = ah + al: Fast2Sum of Kah and sa gh (|Kah| >= gh unless Kah = 0),
  // then the tails
  const float2 ah = fma2(sa, gh, Kah);
  const float2 al = add2(fma2(sa, gh, sub2(Kah, ah)), fma2(sa, gl, Kal));
  // nearest node (magic-number rounding of a 1024 / pi), kept in range
  const float2 jb = fma2(ah, bc(kNodeScale), bc(kMagic));
  const uint32_t j0 = min(__float_as_uint(jb.x) - kMagicBits, (uint32_t)(nodes - 1));
  const uint32_t j1 = min(__float_as_uint(jb.y) - kMagicBits, (uint32_t)(nodes - 1));
  const float2 jf = make_float2((float)j0, (float)j1);
  const TabEntry e0 = tab[j0];
  const TabEntry e1 = tab[j1];
  // d = a - j pi / 1024: the head difference is exact up to one rounding of
  // a value below 2^-9
  const float2 d = add2(fma2(jf, bc(-kNodeH), ah), fma2(jf, bc(-kNodeL), al));
  const float2 f = fma2(fma2(make_float2(e0.sl, e1.sl), d, make_float2(e0.sh, e1.sh)), d,
                        make_float2(e0.cl, e1.cl));
  const float2 ff = floor2(f);
  BinCoord2 c;
  c.fl = add2(make_float2(e0.ch, e1.ch), ff);
  c.fr = sub2(f, ff);
  return c;
}

struct Est2 {
  float2 fl_t, fr_t;   // theta: t = (N - 1) / 2 + h, h = w + 1/2 (floor of h, frac)
  float2 fl_p, fr_p;   // phi:   t directly
};

// tab_t_est / tab_p_est: the tanh map's node tables (unused otherwise).
template <class G>
__device__ __forceinline__ Est2 estimate2(float2 x, float2 y, float2 z, float2 r2h, float2 r2l,
                                          const TabEntry *__restrict__ tab_t_est,
                                          const TabEntry *__restrict__ tab_p_est) {
  constexpr int kN = G::N, kM = G::M;
  Est2 e;
  // theta = atan2(y, x); t = N/2 + w, h = w + 1/2 = K0 + 1/2 + s1 g,
  // g = N beta / (2 pi), beta = atan(min/max of |x|, |y|)
  {
    const float ax0 = fabsf(x.x), ay0 = fabsf(y.x), ax1 = fabsf(x.y), ay1 = fabsf(y.y);
    float2 bh, bl;
    atan_ratio2(make_float2(fminf(ax0, ay0), fminf(ax1, ay1)),
                make_float2(fmaxf(ax0, ay0), fmaxf(ax1, ay1)), bh, bl);
    // psi = beta (|x| >= |y|) or pi/2 - beta; theta = +-psi (x >= 0) or +-(pi - psi)
    const bool u0 = ay0 > ax0, u1 = ay1 > ax1;
    const bool v0 = x.x < 0.0f, v1 = x.y < 0.0f;
    if constexpr (G::MAP == MAP_TANH) {
      // |theta| = Ka + sa beta: Ka = pi/2 (u), pi (v, not u) or 0; sa = -1
      // when u != v; t(theta) = N - t(|theta|) for y < 0 (or -0), the map
      // being odd about theta = 0
      const float2 Kah = make_float2(u0 ? kPi2H : (v0 ? kPiH : 0.0f), u1 ? kPi2H : (v1 ? kPiH : 0.0f));
      const float2 Kal = make_float2(u0 ? kPi2L : (v0 ? kPiL : 0.0f), u1 ? kPi2L : (v1 ? kPiL : 0.0f));
      const float2 sa = make_float2((u0 != v0) ? -1.0f : 1.0f, (u1 != v1) ? -1.0f : 1.0f);
      const BinCoord2 c = tanh_bin2(Kah, Kal, sa, bh, bl, tab_t_est, kTanhNodesT);
      const bool m0 = signbit(y.x), m1 = signbit(y.y);
      // floor t relative to (N - 1) / 2, as the uniform branch returns it
      e.fl_t = make_float2(m0 ? (float)((kN - 1) / 2) - c.fl.x : c.fl.x - (float)((kN - 1) / 2),
                           m1 ? (float)((kN - 1) / 2) - c.fl.y : c.fl.y - (float)((kN - 1) / 2));
      e.fr_t = make_float2(m0 ? 1.0f - c.fr.x : c.fr.x, m1 ? 1.0f - c.fr.y : c.fr.y);
    } else {
    // u: psi = pi/2 - beta (offset N/4, sign -); v: pi - psi (offset N/2 - ., sign
    // flips); y < 0 (or -0): theta = -(.) (offset and sign flip)
    float2 K0 = make_float2(u0 ? 0.25f * (float)kN : 0.0f, u1 ? 0.25f * (float)kN : 0.0f);
    K0 = make_float2(v0 ? 0.5f * (float)kN - K0.x : K0.x, v1 ? 0.5f * (float)kN - K0.y : K0.y);
    K0 = make_float2(copysignf(K0.x, y.x), copysignf(K0.y, y.y));
    // s1 = (u != v ? -1 : 1), negated again for y < 0 (sign-bit xor)
    const float2 s1 =
        make_float2(__uint_as_float(__float_as_uint((u0 != v0) ? -1.0f : 1.0f) ^
                                    (__float_as_uint(y.x) & 0x80000000u)),
                    __uint_as_float(__float_as_uint((u1 != v1) ? -1.0f : 1.0f) ^
                                    (__float_as_uint(y.y) & 0x80000000u)));
    const BinCoord2 c = bin_coord2(add2(K0, bc(0.5f)), s1, bh, bl, G::CTH, G::CTL);
    e.fl_t = c.fl;
    e.fr_t = c.fr;
    }
  }
  // phi = atan2(rho, z); t = K0 + s1 g, g = M beta / pi
  {
    // rho = sqrt(x^2 + y^2): one Newton step on the float-float sum (relative
    // error 2^-24, 0.0012 bin); 0 stays about 1e-18
    const float2 rr = make_float2(fmaxf(r2h.x, 1e-36f), fmaxf(r2h.y, 1e-36f));
    const float2 yr = make_float2(rsqrtf(rr.x), rsqrtf(rr.y));
    const float2 q0 = mul2(rr, yr);
    const float2 rho = fma2(add2(fma2(neg2(q0), q0, rr), r2l), mul2(yr, bc(0.5f)), q0);
    const float rho0 = rho.x, rho1 = rho.y;
    const float az0 = fabsf(z.x), az1 = fabsf(z.y);
    float2 bh, bl;
    atan_ratio2(make_float2(fminf(az0, rho0), fminf(az1, rho1)),
                make_float2(fmaxf(az0, rho0), fmaxf(az1, rho1)), bh, bl);
    const bool u0 = rho0 > az0, u1 = rho1 > az1;
    const bool n0 = z.x < 0.0f, n1 = z.y < 0.0f;
    if constexpr (G::MAP == MAP_TANH) {
      // phi' = min(phi, pi - phi) = pi/2 - beta (rho > |z|) or beta; t(phi) =
      // M - t(phi') for z < 0, the map being odd about phi = pi/2
      const float2 Kah = make_float2(u0 ? kPi2H : 0.0f, u1 ? kPi2H : 0.0f);
      const float2 Kal = make_float2(u0 ? kPi2L : 0.0f, u1 ? kPi2L : 0.0f);
      const float2 sa = make_float2(u0 ? -1.0f : 1.0f, u1 ? -1.0f : 1.0f);
      const BinCoord2 c = tanh_bin2(Kah, Kal, sa, bh, bl, tab_p_est, kTanhNodesP);
      e.fl_p = make_float2(n0 ? (float)(kM - 1) - c.fl.x : c.fl.x,
                           n1 ? (float)(kM - 1) - c.fl.y : c.fl.y);
      e.fr_p = make_float2(n0 ? 1.0f - c.fr.x : c.fr.x, n1 ? 1.0f - c.fr.y : c.fr.y);
    } else {
    // |z| >= rho: t = g (z >= 0) or M - g;  rho > |z|: t = M/2 -+ g
    const float2 K0 = make_float2(u0 ? 0.5f * (float)kM : (n0 ? (float)kM : 0.0f),
                                  u1 ? 0.5f * (float)kM : (n1 ? (float)kM : 0.0f));
    const float2 s1 = make_float2((u0 != n0) ? -1.0f : 1.0f, (u1 != n1) ? -1.0f : 1.0f);
    const BinCoord2 c = bin_coord2(K0, s1, bh, bl, G::CPH, G::CPL);
    e.fl_p = c.fl;
    e.fr_p = c.fr;
    }
  }
  return e;
}

// Error-free side test for one pending decision (generic tables and FP64
// fallback): kind 0 the theta boundary k + 1/2, kind 1 the phi boundary.
// One straight path for both kinds.
template <class G>
__device__ __forceinline__ int exact_side(int kind, int k, float xs, float ys, float zs,
                                          const DevFormat &F, const TabEntry *tab_t,
                                          const TabEntry *tab_p) {
  const bool ph = kind != 0;
  FF c, s;
  if constexpr (G::MAP == MAP_TANH) {
    // signed cos/sin of the boundary angle from the per-boundary tables
    const TabEntry e = ph ? F.bnd_p[k] : F.bnd_t[k];
    c = FF{e.ch, e.cl};
    s = FF{e.sh, e.sl};
  } else {
    bool cn, sn;
    sincospi_grid(ph ? 2 * k + 1 : 2 * k + 1 - F.N, ph ? F.Dp : F.Dt, ph ? tab_p : tab_t,
                  ph ? F.sp : F.st, ph ? F.Kp_h : F.Kt_h, ph ? F.Kp_l : F.Kt_l, c, s, cn, sn);
    c = neg_if(c, cn);
    s = neg_if(s, sn);
  }
  // theta: sign(y cos - x sin);  phi: sign(rho cos - z sin)
  float a = ys, a_l = 0.0f;
  if (ph) {
    const float px = xs * xs, ex = fmaf(xs, xs, -px);
    const float py = ys * ys, ey = fmaf(ys, ys, -py);
    const float r2h = px + py;
    const float t = r2h - px;
    const float r2l = ((px - (r2h - t)) + (py - t)) + (ex + ey);
    float rho_h = 0.0f, rho_l = 0.0f;
    if (r2h > 0.0f) {
      const float y1 = rsqrtf(r2h);
      const float hy1 = 0.5f * y1;
      const float q0 = r2h * y1;
      rho_h = fmaf(fmaf(-q0, q0, r2h) + r2l, hy1, q0);
      rho_l = (fmaf(-rho_h, rho_h, r2h) + r2l) * hy1;
    }
    a = rho_h;
    a_l = rho_l;
  }
  const int side = side_ge(a, a_l, c, ph ? zs : xs, s);
  if (side >= 0) return side;
  return ph ? side_phi_exact<G::MAP>(xs, ys, zs, k, F)
            : side_theta_exact<G::MAP>(xs, ys, k, F);
}

template <int MAP>
static __device__ __noinline__ uint64_t encode_generic(float x, float y, float z, const DevFormat &F,
                                                       const TabEntry *tab_t,
                                                       const TabEntry *tab_p, uint32_t &flags) {
  return encode_vec<MAP>(x, y, z, F, tab_t, tab_p, flags);
}

template <int MAP>
static __device__ __noinline__ float3 decode_generic(uint64_t w, const DevFormat &F, const TabEntry *tab_t,
                                              const TabEntry *tab_p) {
  return decode_word<MAP>(w, F, tab_t, tab_p);
}

// Result of encode2 for two vectors: provisional words and what the deferred
// exact tests need.
struct Enc2 {
  uint64_t w0, w1;         // words (provisional where pend != 0)
  uint32_t pend0, pend1;   // pending: bit 0 theta test, bit 1 phi test, bit 2 generic encode
  int nt0, nt1, np0, np1;  // k of a pending kind, else the code
  uint32_t hi0, hi1;       // high words without the n_phi bits
};

// Encodes two vectors.  The word of a vector with a pending exact decision,
// or outside the fast path's magnitude window (zero, tiny, huge, Inf, NaN:
// the generic encoder, with its range handling and events), is provisional:
// the caller queues it with push2.  est (optional) receives the angle
// estimates.  REUSE: the vectors are positive multiples RN(rho v) of vectors
// v whose estimates est holds; those stand for the angle estimates here,
// with the ambiguity band widened by kReuseEps, and an element with force set
// (rho not positive and finite, or v outside the window) goes to the generic
// encoder.
template <class G, bool REUSE = false>
__device__ __forceinline__ Enc2 encode2(float2 x, float2 y, float2 z, const DevFormat &F,
                                        const TabEntry *__restrict__ tab_t,
                                        const TabEntry *__restrict__ tab_p,
                                        Est2 *est = nullptr, bool force0 = false,
                                        bool force1 = false) {
  constexpr int kN = G::N, kM = G::M;
  Enc2 r;
  // squares and sums in float-float
  const float2 px = mul2(x, x), ex = fma2(x, x, neg2(px));
  const float2 py = mul2(y, y), ey = fma2(y, y, neg2(py));
  const float2 pz = mul2(z, z), ez = fma2(z, z, neg2(pz));
  const float2 r2h = add2(px, py);
  float2 t = sub2(r2h, px);
  const float2 r2l = add2(add2(sub2(px, sub2(r2h, t)), sub2(py, t)), add2(ex, ey));
  const float2 sh = add2(r2h, pz);
  t = sub2(sh, r2h);
  const float2 sl = add2(add2(sub2(r2h, sub2(sh, t)), sub2(pz, t)), add2(r2l, ez));
  // |x|^2 in [2^-64, 2^64): NaN, Inf, the zero vector and magnitudes the
  // fast path does not serve fail the test
  const bool gen0 = !(sh.x >= 0x1p-64f && sh.x < 0x1p64f);
  const bool gen1 = !(sh.y >= 0x1p-64f && sh.y < 0x1p64f);
  // float-float square root, RN32
  const float2 y0 = make_float2(rsqrtf(sh.x), rsqrtf(sh.y));
  const float2 hy0 = mul2(y0, bc(0.5f));
  const float2 q0 = mul2(sh, y0);
  const float2 rh = fma2(add2(fma2(neg2(q0), q0, sh), sl), hy0, q0);
  const float2 rl = mul2(add2(fma2(neg2(rh), rh, sh), sl), hy0);
  float2 r32 = add2(rh, rl);
  const float2 dev = add2(sub2(rh, r32), rl);
  bool nslow0, nslow1;
  {
    const float hu0 = __uint_as_float((__float_as_uint(r32.x) & 0x7f800000u) - (24u << 23));
    const float hu1 = __uint_as_float((__float_as_uint(r32.y) & 0x7f800000u) - (24u << 23));
    nslow0 = (hu0 - fabsf(dev.x) <= kNormAmbig * r32.x) || ((__float_as_uint(r32.x) & 0x7fffffu) == 0u);
    nslow1 = (hu1 - fabsf(dev.y) <= kNormAmbig * r32.y) || ((__float_as_uint(r32.y) & 0x7fffffu) == 0u);
  }
  // a magnitude within the norm's error bound of an FP32 rounding boundary
  // (about 2^-18 of the vectors) is settled by the generic encoder, through
  // the queue like the out-of-window vectors
  const bool gq0 = gen0 || nslow0 || (REUSE && force0);
  const bool gq1 = gen1 || nslow1 || (REUSE && force1);
  // angle estimates
  Est2 e;
  if constexpr (REUSE) {
    e = *est;
  } else {
    e = estimate2<G>(x, y, z, r2h, r2l, tab_t, tab_p);
    if (est) *est = e;
  }
  // k = floor(t) clamped to [0, n_max - 1]; the fraction absorbs the clamp
  // (t = n_max gives fraction 1, t < 0 a negative one: never flagged)
  float2 ft = add2(e.fl_t, bc((float)((kN - 1) / 2)));
  const float2 ftc = make_float2(fminf(fmaxf(ft.x, 0.0f), (float)(kN - 1)),
                                 fminf(fmaxf(ft.y, 0.0f), (float)(kN - 1)));
  const float2 frt = add2(e.fr_t, sub2(ft, ftc));
  const float2 fpc = make_float2(fminf(fmaxf(e.fl_p.x, 0.0f), (float)(kM - 1)),
                                 fminf(fmaxf(e.fl_p.y, 0.0f), (float)(kM - 1)));
  const float2 frp = add2(e.fr_p, sub2(e.fl_p, fpc));
  const int kt0 = (int)(__float_as_uint(ftc.x + kMagic) - kMagicBits);
  const int kt1 = (int)(__float_as_uint(ftc.y + kMagic) - kMagicBits);
  const int kp0 = (int)(__float_as_uint(fpc.x + kMagic) - kMagicBits);
  const int kp1 = (int)(__float_as_uint(fpc.y + kMagic) - kMagicBits);
  int nt0 = kt0 + (frt.x >= 0.5f ? 1 : 0), nt1 = kt1 + (frt.y >= 0.5f ? 1 : 0);
  int np0 = kp0 + (frp.x >= 0.5f ? 1 : 0), np1 = kp1 + (frp.y >= 0.5f ? 1 : 0);
  // pending exact decisions: kinds within kEps of a rounding boundary
  // (bit 0 theta, bit 1 phi); their words are provisional
  constexpr float eps = (G::MAP == MAP_TANH ? kEpsTanh : kEps) + (REUSE ? kReuseEps : 0.0f);
  r.pend0 = gq0 ? 4u : (fabsf(frt.x - 0.5f) <= eps ? 1u : 0u) | (fabsf(frp.x - 0.5f) <= eps ? 2u : 0u);
  r.pend1 = gq1 ? 4u : (fabsf(frt.y - 0.5f) <= eps ? 1u : 0u) | (fabsf(frp.y - 0.5f) <= eps ? 2u : 0u);
  r.nt0 = (r.pend0 & 1u) ? kt0 : nt0;
  r.nt1 = (r.pend1 & 1u) ? kt1 : nt1;
  r.np0 = (r.pend0 & 2u) ? kp0 : np0;
  r.np1 = (r.pend1 & 2u) ? kp1 : np1;
  // canonical forms and packing (Fig. manbit)
  if (nt0 == kN || np0 == 0 || np0 == kM) nt0 = 0;
  if (nt1 == kN || np1 == 0 || np1 == kM) nt1 = 0;
  const uint32_t rb0 = __float_as_uint(r32.x), rb1 = __float_as_uint(r32.y);
  r.hi0 = G::hi_of(rb0);
  r.hi1 = G::hi_of(rb1);
  r.w0 = G::pack(r.hi0, np0, nt0);
  r.w1 = G::pack(r.hi1, np1, nt1);
  return r;
}

// ---------------------------------------------------- deferred exact tests
// A vector whose bin coordinate lies within kEps of a rounding boundary gets
// a provisional word; its exact side-of-boundary tests run later from a
// per-warp queue in shared memory, one item per lane, 32 at a time, and the
// final word overwrites the provisional one (same warp, ordered by
// __syncwarp).  Capacity: at most 31 items wait between pushes and one push
// adds at most 64.
constexpr int kQueueCap = 95;

struct PendItem {
  uint64_t *dst;   // word to overwrite
  float x, y, z;   // the encoded vector
  uint32_t hi;     // high word without the n_phi bits
  int nt;          // theta: k when pending, else the code
  uint32_t npp;    // phi: k when pending, else the code (bits 0..28); pending bits (29..31)
};

// Range events of the generic encoder, per thread (bit 0 overflow, 1
// underflow, 2 NaN of its flags).
struct Events {
  uint32_t o = 0, u = 0, q = 0;
  __device__ __forceinline__ void add(uint32_t flags) {
    o += flags & 1u;
    u += (flags >> 1) & 1u;
    q += (flags >> 2) & 1u;
  }
};

struct WarpQueue {
  PendItem *q;     // this warp's slots
  int count;       // warp-uniform
};

__device__ __forceinline__ WarpQueue warp_queue(void *base) {
  WarpQueue wq;
  wq.q = reinterpret_cast<PendItem *>(base) + (threadIdx.x >> 5) * kQueueCap;
  wq.count = 0;
  return wq;
}

// Runs once per 32 queued items: kept out of line so that the main loop's
// register allocation does not carry the exact test or the generic encoder.
// Returns the generic encoder's range events (0 for an exact test).
template <class G>
static __device__ __noinline__ uint32_t resolve_item(const PendItem *pit, const DevFormat &F,
                                                     const TabEntry *tab_t,
                                                     const TabEntry *tab_p) {
  const PendItem it = *pit;
  const uint32_t pend = it.npp >> 29;
  if (pend & 4u) {
    uint32_t flags = 0;
    *it.dst = encode_generic<G::MAP>(it.x, it.y, it.z, F, tab_t, tab_p, flags);
    return flags;
  }
  int nt = it.nt;
  int np = (int)(it.npp & 0x1FFFFFFFu);
  // one kind-agnostic test per item; a second only when both kinds wait
  const int kind = (pend & 1u) ? 0 : 1;
  const int side = exact_side<G>(kind, kind ? np : nt, it.x, it.y, it.z, F, tab_t, tab_p);
  if (kind == 0) nt += side;
  else np += side;
  if (pend == 3u) np += exact_side<G>(1, np, it.x, it.y, it.z, F, tab_t, tab_p);
  if (nt == G::N || np == 0 || np == G::M) nt = 0;
  *it.dst = G::pack(it.hi, np, nt);
  return 0u;
}

// Queues the pending vectors of one encode2 result (element 0 -> dst0,
// element 1 -> dst0 + 1; inactive lanes queue nothing) and resolves full
// batches.  All lanes of the warp call it.
template <class G>
__device__ __forceinline__ void push2(WarpQueue &wq, bool act, const Enc2 &e, float2 x, float2 y,
                                      float2 z, uint64_t *dst0, const DevFormat &F,
                                      const TabEntry *tab_t, const TabEntry *tab_p,
                                      Events *ev = nullptr) {
  const uint32_t p0 = act ? e.pend0 : 0u, p1 = act ? e.pend1 : 0u;
  const unsigned b0 = __ballot_sync(0xffffffffu, p0 != 0u);
  const unsigned b1 = __ballot_sync(0xffffffffu, p1 != 0u);
  if ((b0 | b1) == 0u) return;
  const unsigned lt = (1u << (threadIdx.x & 31)) - 1u;
  int slot = wq.count + __popc(b0 & lt) + __popc(b1 & lt);
  if (p0) {
    wq.q[slot++] = PendItem{dst0, x.x, y.x, z.x, e.hi0, e.nt0, (uint32_t)e.np0 | (p0 << 29)};
  }
  if (p1) {
    wq.q[slot] = PendItem{dst0 + 1, x.y, y.y, z.y, e.hi1, e.nt1, (uint32_t)e.np1 | (p1 << 29)};
  }
  wq.count += __popc(b0) + __popc(b1);
  while (wq.count >= 32) {
    __syncwarp();
    const uint32_t fl = resolve_item<G>(wq.q + wq.count - 32 + (threadIdx.x & 31), F, tab_t, tab_p);
    if (ev) ev->add(fl);
    wq.count -= 32;
    __syncwarp();
  }
}

// Resolves what is left in the queue (all lanes call it).
template <class G>
__device__ __forceinline__ void drain(WarpQueue &wq, const DevFormat &F, const TabEntry *tab_t,
                                      const TabEntry *tab_p, Events *ev = nullptr) {
  if (wq.count == 0) return;
  __syncwarp();
  if ((int)(threadIdx.x & 31) < wq.count) {
    const uint32_t fl = resolve_item<G>(wq.q + (threadIdx.x & 31), F, tab_t, tab_p);
    if (ev) ev->add(fl);
  }
  wq.count = 0;
  __syncwarp();
}

// 16-byte asynchronous global-to-shared copy (L2 only).
__device__ __forceinline__ void cp_async16(float4 *dst, const void *src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(
                   (uint32_t)__cvta_generic_to_shared(dst)),
               "l"(__cvta_generic_to_global(src))
               : "memory");
}

// Starts the copies of the tanh map's per-code table entries of a word pair
// into the shared-memory slots dst[0], dst[ss], dst[2 ss], dst[3 ss] (any
// field values index inside the tables: n_theta <= N, n_phi <= M).
template <class G>
__device__ __forceinline__ void stage_entries(uint64_t w0, uint64_t w1, const DevFormat &F,
                                              float4 *dst, int ss) {
  uint32_t nt0, np0, nt1, np1;
  G::unpack((uint32_t)(w0 >> 32), (uint32_t)w0, nt0, np0);
  G::unpack((uint32_t)(w1 >> 32), (uint32_t)w1, nt1, np1);
  cp_async16(dst, F.dec_t + nt0);
  cp_async16(dst + ss, F.dec_t + nt1);
  cp_async16(dst + 2 * ss, F.dec_p + np0);
  cp_async16(dst + 3 * ss, F.dec_p + np1);
}
// The per-code phi^ entries of a word pair into slots 2 ss and 3 ss.
template <class G>
__device__ __forceinline__ void stage_phi(uint64_t w0, uint64_t w1, const DevFormat &F,
                                          float4 *dst, int ss) {
  uint32_t nt0, np0, nt1, np1;
  G::unpack((uint32_t)(w0 >> 32), (uint32_t)w0, nt0, np0);
  G::unpack((uint32_t)(w1 >> 32), (uint32_t)w1, nt1, np1);
  cp_async16(dst + 2 * ss, F.phi_tab + min((int)np0, G::M - (int)np0));
  cp_async16(dst + 3 * ss, F.phi_tab + min((int)np1, G::M - (int)np1));
}

// Decodes two words through the fast path, falling back per element.  PT:
// F.phi_tab holds the per-code phi^ table.  stg: the tanh map's entries,
// staged.
template <class G, bool PT = true>
__device__ __forceinline__ void decode2_full(uint64_t w0, uint64_t w1, const DevFormat &F,
                                             const TabEntry *tab_t, const TabEntry *tab_p,
                                             float2 &X, float2 &Y, float2 &Z,
                                             const Staged *stg = nullptr) {
  bool s0, s1;
  decode2<G, PT>(w0, w1, F, tab_t, tab_p, X, Y, Z, s0, s1, stg);
  if (s0) {
    const float3 v = decode_generic<G::MAP>(w0, F, tab_t, tab_p);
    X.x = v.x; Y.x = v.y; Z.x = v.z;
  }
  if (s1) {
    const float3 v = decode_generic<G::MAP>(w1, F, tab_t, tab_p);
    X.y = v.x; Y.y = v.y; Z.y = v.z;
  }
}

// Shared-memory tables of the fast kernels: the uniform head tables, or for
// the tanh map the encoder's node tables; the deferred-test queues follow.
template <class G>
__host__ __device__ __forceinline__ int fast_ntab_t(const DevFormat &F) {
  return G::MAP == MAP_TANH ? F.nest_t : F.nent_t;
}
template <class G>
__host__ __device__ __forceinline__ int fast_ntab(const DevFormat &F) {
  return G::MAP == MAP_TANH ? F.nest_t + F.nest_p : F.nent_t + F.nent_p;
}
template <class G>
__device__ __forceinline__ void stage_fast_tables(const DevFormat &F, TabEntry *smem) {
  const float4 *src = reinterpret_cast<const float4 *>(G::MAP == MAP_TANH ? F.est_tab : F.tab);
  float4 *dst = reinterpret_cast<float4 *>(smem);
  const int total = fast_ntab<G>(F);
  for (int i = threadIdx.x; i < total; i += blockDim.x) dst[i] = __ldg(src + i);
  __syncthreads();
}

}  // namespace fast
}  // namespace ivc
