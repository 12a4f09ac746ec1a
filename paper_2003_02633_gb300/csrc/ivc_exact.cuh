// Exact-decision arithmetic of the codec in 64- and 128-bit integers (no
// floating point wider than FP32 on the device).
//
// The FP32 paths of ivc_device.cuh and ivc_fast.cuh settle every rounding
// decision of the method whose operands lie farther than their error bound
// from the boundary (about 2^-40 relative).  The remaining ones come here:
//   * magnitude (Sec. 2.3): RN32 of sqrt(x^2 + y^2 + z^2) decided by the
//     exact sign of S - m^2 at the FP32 rounding midpoints m around the
//     candidate, in 128-bit integers (no error at all);
//   * angles (Eq. a_disc): the side of the boundary direction on which the
//     input lies, sign(y cos t - x sin t) or sign(rho cos p - z sin p), from
//     cos/sin of the boundary angle to about 2^-57 relative;
//   * decode (Eq. a_inv, cart2sphere): r cos(theta^) sin(phi^) etc. to about
//     2^-56 relative, rounded away from zero.
// Values are unsigned "SF" numbers: a 64-bit mantissa normalised to bit 63
// and a binary exponent, with a flag telling whether the value is exact.
// cos and sin of pi b / (2D) on [0, pi/4] come from Taylor series evaluated
// in Q1.63 fixed point; the angle itself is b times pi / (2D), the latter
// precomputed on the host from floor(pi 2^126) by integer division.  The
// Niven values on that range (b = 0: cos 1, sin 0; 3b = D: sin 1/2) are
// exact, so results that are exactly representable (poles, axes, halves) are
// rounded exactly; every other value involved is irrational and lies at
// least the error bound away from an FP32 grid point except with probability
// about 2^-16 of the cases that reach this code.
#pragma once
#include <cmath>
#include <cstdint>
#include <cstring>

namespace ivc {
namespace exact {

struct SF {
  uint64_t m;   // bit 63 set, or 0 for the value zero
  int e;        // value = m 2^e
  bool exact;   // no rounding happened on the way
};

__host__ __device__ __forceinline__ int clz64(uint64_t v) {
#ifdef __CUDA_ARCH__
  return __clzll((long long)v);
#else
  return v ? __builtin_clzll(v) : 64;
#endif
}

__host__ __device__ __forceinline__ uint64_t mulhi64(uint64_t a, uint64_t b) {
#ifdef __CUDA_ARCH__
  return __umul64hi(a, b);
#else
  return (uint64_t)(((unsigned __int128)a * b) >> 64);
#endif
}

__host__ __device__ __forceinline__ SF sf_norm(uint64_t m, int e, bool exact) {
  if (m == 0) return SF{0ull, 0, exact};
  const int z = clz64(m);
  return SF{m << z, e - z, exact};
}

__host__ __device__ __forceinline__ SF sf_from_u64(uint64_t v) { return sf_norm(v, 0, true); }

// |v| for a finite FP32 v.
__host__ __device__ __forceinline__ SF sf_from_float(float v) {
  uint32_t b;
  memcpy(&b, &v, 4);
  b &= 0x7fffffffu;
  const uint32_t E = b >> 23, man = b & 0x7fffffu;
  if (E == 0) return sf_norm(man, -149, true);
  return sf_norm((uint64_t)(man | 0x800000u), (int)E - 150, true);
}

__host__ __device__ __forceinline__ SF sf_mul(SF a, SF b) {
  if (a.m == 0 || b.m == 0) {
    // an exact zero makes the product an exact zero
    const bool ex = (a.m == 0 && a.exact) || (b.m == 0 && b.exact) || (a.exact && b.exact);
    return SF{0ull, 0, ex};
  }
  const uint64_t hi = mulhi64(a.m, b.m), lo = a.m * b.m;
  int e = a.e + b.e + 64;
  bool ex = a.exact && b.exact;
  uint64_t m;
  if (hi >> 63) {
    m = hi;
    ex = ex && lo == 0ull;
  } else {
    m = (hi << 1) | (lo >> 63);
    e -= 1;
    ex = ex && (lo << 1) == 0ull;
  }
  return SF{m, e, ex};
}

// a + b for a, b >= 0 (truncated to 64 bits).
__host__ __device__ __forceinline__ SF sf_add(SF a, SF b) {
  if (a.m == 0) return SF{b.m, b.e, a.exact && b.exact};
  if (b.m == 0) return SF{a.m, a.e, a.exact && b.exact};
  if (a.e < b.e) {
    const SF t = a;
    a = b;
    b = t;
  }
  const int d = a.e - b.e;
  uint64_t bm = 0;
  bool lost = false;
  if (d >= 64) {
    lost = true;
  } else if (d > 0) {
    bm = b.m >> d;
    lost = (b.m << (64 - d)) != 0ull;
  } else {
    bm = b.m;
  }
  uint64_t s = a.m + bm;
  int e = a.e;
  bool ex = a.exact && b.exact && !lost;
  if (s < a.m) {  // carry out of bit 63
    ex = ex && (s & 1ull) == 0ull;
    s = (s >> 1) | 0x8000000000000000ull;
    e += 1;
  }
  return SF{s, e, ex};
}

// Sign of a - b (both >= 0) from the represented values.
__host__ __device__ __forceinline__ int sf_cmp(SF a, SF b) {
  if (a.m == 0 || b.m == 0) {
    if (a.m == 0 && b.m == 0) return 0;
    return a.m == 0 ? -1 : 1;
  }
  if (a.e != b.e) return a.e > b.e ? 1 : -1;
  if (a.m != b.m) return a.m > b.m ? 1 : -1;
  return 0;
}

// Integer significand and exponent of a finite FP32 magnitude: |v| = V 2^(ev - 23).
__host__ __device__ __forceinline__ void f32_parts(float v, uint32_t &V, int &ev) {
  uint32_t b;
  memcpy(&b, &v, 4);
  b &= 0x7fffffffu;
  const uint32_t E = b >> 23;
  V = (b & 0x7fffffu) | (E ? 0x800000u : 0u);
  ev = E ? (int)E - 127 : -126;
}

// |h + l| for a float-float value (|l| below |h|, or h = 0), with its sign.
__host__ __device__ inline SF sf_from_ff(float h, float l, bool &neg) {
  uint32_t hb, lb;
  memcpy(&hb, &h, 4);
  memcpy(&lb, &l, 4);
  if ((hb & 0x7fffffffu) == 0u) {
    neg = (lb >> 31) != 0u && (lb & 0x7fffffffu) != 0u;
    return sf_from_float(l);
  }
  neg = (hb >> 31) != 0u;
  if ((lb & 0x7fffffffu) == 0u) return sf_from_float(h);
  uint32_t Hm, Lm;
  int eh, el;
  f32_parts(h, Hm, eh);
  f32_parts(l, Lm, el);
  const int d = eh - el;  // >= 0
  if (d > 100) {
    SF r = sf_from_float(h);
    r.exact = false;
    return r;
  }
  // |h + l| = ((Hm << d) +- Lm) 2^(el - 23), positive since |l| < |h|
  const unsigned __int128 hv = (unsigned __int128)Hm << d;
  const unsigned __int128 v = (((hb ^ lb) >> 31) == 0u) ? hv + Lm : hv - Lm;
  const uint64_t top = (uint64_t)(v >> 64), low = (uint64_t)v;
  const int nbits = top ? 128 - clz64(top) : 64 - clz64(low);
  if (nbits <= 64) return sf_norm(low, el - 23, true);
  const int sh = nbits - 64;
  const uint64_t m = (uint64_t)(v >> sh);
  const bool lost = (v & (((unsigned __int128)1 << sh) - 1)) != 0;
  return SF{m, el - 23 + sh, !lost};
}

// pi / den as m 2^e with a 64-bit m (bit 63 set), truncated: floor(pi 2^126)
// divided by den in exact integer arithmetic (host set-up of the formats), so
// every host gives the same bits.
inline void pi_over_host(long long den, uint64_t &m, int32_t &e) {
  const unsigned __int128 pi126 =
      ((unsigned __int128)0xC90FDAA22168C234ull << 64) | (unsigned __int128)0xC4C6628B80DC1CD1ull;
  const unsigned __int128 q = pi126 / (unsigned __int128)den;
  int nb = 128;
  while (nb > 64 && ((q >> (nb - 1)) & 1u) == 0u) --nb;
  m = (uint64_t)(q >> (nb - 64));
  e = -126 + (nb - 64);
}

// ----------------------------------------------------- Q1.63 fixed point
constexpr uint64_t kQOne = 1ull << 63;

__host__ __device__ __forceinline__ uint64_t qmul(uint64_t a, uint64_t b) {
  const uint64_t hi = mulhi64(a, b), lo = a * b;
  return (hi << 1) | (lo >> 63);
}

// 1 / (k (k + 1)) in Q1.63 (truncated), k = 1 .. 19
__host__ __device__ __forceinline__ uint64_t inv_pair(int k) {
  return kQOne / (uint64_t)(k * (k + 1));
}

// cos and sin of the folded angle pi b / (2D), b in [0, D/2]; Kpi = pi / (2D).
__host__ __device__ inline void sincos_folded(int b, int D, SF Kpi, SF &c, SF &s) {
  if (b == 0) {
    c = SF{kQOne, -63, true};
    s = SF{0ull, 0, true};
    return;
  }
  const SF alpha = sf_mul(Kpi, sf_from_u64((uint64_t)b));  // < pi / 4
  // alpha in Q1.63 (alpha < 1: shift right by -(e + 63) >= 1)
  const int sh = -(alpha.e + 63);
  const uint64_t aq = sh >= 64 ? 0ull : alpha.m >> sh;
  const uint64_t x = qmul(aq, aq);  // alpha^2 < 0.62
  // sin(alpha) = alpha (1 - x/(2.3) (1 - x/(4.5) (... (1 - x/(18.19)))))
  uint64_t t = kQOne;
#pragma unroll
  for (int k = 18; k >= 2; k -= 2) t = kQOne - qmul(qmul(x, inv_pair(k)), t);
  // cos(alpha) = 1 - x/(1.2) (1 - x/(3.4) (... (1 - x/(19.20))))
  uint64_t u = kQOne;
#pragma unroll
  for (int k = 19; k >= 1; k -= 2) u = kQOne - qmul(qmul(x, inv_pair(k)), u);
  c = sf_norm(u, -63, false);
  if (3 * b == D) {
    s = SF{kQOne, -64, true};  // sin(pi / 6) = 1/2
  } else {
    s = sf_mul(alpha, sf_norm(t, -63, false));
  }
}

// cos and sin (magnitudes and signs) of pi m / D, m in [-D, D], by the exact
// integer fold onto [0, pi/4].
__host__ __device__ inline void sincospi_grid(int m, int D, SF Kpi, SF &c, SF &s, bool &cneg,
                                              bool &sneg) {
  sneg = m < 0;
  const int a = m < 0 ? -m : m;
  cneg = 2 * a > D;
  const int a1 = cneg ? D - a : a;
  const bool swap = 4 * a1 > D;
  const int b = swap ? D - 2 * a1 : 2 * a1;
  SF cc, ss;
  sincos_folded(b, D, Kpi, cc, ss);
  c = swap ? ss : cc;
  s = swap ? cc : ss;
  // an exact zero carries no sign
  if (c.m == 0) cneg = false;
  if (s.m == 0) sneg = false;
}

// Round a value >= 0 away from zero to FP32 (the value itself when exact and
// representable); subnormal results keep the same rule, values beyond the
// FP32 range give infinity.
__host__ __device__ inline float ra32(SF v) {
  if (v.m == 0) return 0.0f;
  // value = m 2^e = 1.f 2^(e + 63)
  int E = v.e + 63 + 127;  // biased exponent of the leading bit
  uint64_t q;
  bool rest;
  if (E >= 1) {
    q = v.m >> 40;  // 24 bits
    rest = (v.m & ((1ull << 40) - 1ull)) != 0ull || !v.exact;
  } else {
    const int sh = 40 + (1 - E);  // subnormal: fewer bits
    q = sh >= 64 ? 0ull : v.m >> sh;
    rest = (sh >= 64 ? v.m != 0ull : (v.m & ((1ull << sh) - 1ull)) != 0ull) || !v.exact;
    E = 0;
  }
  if (rest) {
    q += 1;
    if (E >= 1 && q == (1ull << 24)) {
      q >>= 1;
      E += 1;
    } else if (E == 0 && q == (1ull << 23)) {
      E = 1;  // rounded up into the normal range (q keeps its implicit bit)
    }
  }
  if (E >= 255) {
    const uint32_t inf = 0x7f800000u;
    float f;
    memcpy(&f, &inf, 4);
    return f;
  }
  const uint32_t bits = E >= 1 ? ((uint32_t)E << 23) | ((uint32_t)q & 0x7fffffu) : (uint32_t)q;
  float f;
  memcpy(&f, &bits, 4);
  return f;
}

// Sign decision of (sa ? -A : A) - (sb ? -B : B) >= 0 for magnitudes A, B.
__host__ __device__ __forceinline__ int side_of(SF A, bool sa, SF B, bool sb) {
  if (A.m == 0) sa = false;
  if (B.m == 0) sb = false;
  if (!sa && sb) return 1;
  if (sa && !sb) return (A.m == 0 && B.m == 0) ? 1 : 0;
  const int c = sf_cmp(A, B);  // same signs
  return sa ? (c <= 0 ? 1 : 0) : (c >= 0 ? 1 : 0);
}

// Sign of x^2 + y^2 + z^2 - m^2, m = M 2^-25 a rounding midpoint of the
// scaled norm, for components sorted a >= b >= c with a in [1, 2):
// a = A 2^-23, b = B 2^(eb - 23), c = C 2^(ec - 23) (B, C may be 0).
// U = a^2 - m^2 = (a - m)(a + m) is a multiple of 2^-50 with |U| > 2^-25
// (a - m is a nonzero multiple of 2^-25); the smaller squares join it in
// exact 128-bit sums whenever they can change its sign.
__host__ __device__ inline int sign_s_minus_m2(uint32_t A, uint32_t B, int eb, uint32_t C, int ec,
                                               uint64_t M) {
  const long long U = 16ll * (long long)((uint64_t)A * A) - (long long)(M * M);  // units 2^-50
  if (B == 0u || eb < -13) return U > 0 ? 1 : -1;  // b^2 + c^2 < 2^-25 < |U|
  const int L2 = 46 - 2 * eb > 50 ? 46 - 2 * eb : 50;  // unit 2^-L2 holds U and b^2
  if (C == 0u || 2 * ec + 2 <= -L2) {
    // c^2 < 2^-L2: it decides only an exact zero of U + b^2
    __int128 T = (__int128)U << (L2 - 50);
    T += (__int128)((uint64_t)B * B) << (2 * eb - 46 + L2);
    if (T != 0) return T > 0 ? 1 : -1;
    return C != 0u ? 1 : 0;
  }
  const int L3 = 46 - 2 * ec > 50 ? 46 - 2 * ec : 50;  // <= 120 here
  __int128 T = (__int128)U << (L3 - 50);
  T += (__int128)((uint64_t)B * B) << (2 * eb - 46 + L3);
  T += (__int128)((uint64_t)C * C) << (2 * ec - 46 + L3);
  return T > 0 ? 1 : (T < 0 ? -1 : 0);
}

// RN32 of sqrt(xs^2 + ys^2 + zs^2) for components scaled so that the largest
// magnitude lies in [1, 2), given a candidate r32 that is the correctly
// rounded norm or an FP32 neighbour of it.  Exact (ties to even).
__host__ __device__ inline float norm_rn(float xs, float ys, float zs, float r32) {
  float a = fabsf(xs), b = fabsf(ys), c = fabsf(zs);
  if (a < b) { const float t = a; a = b; b = t; }
  if (b < c) { const float t = b; b = c; c = t; }
  if (a < b) { const float t = a; a = b; b = t; }
  uint32_t A, B, C;
  int ea, eb, ec;
  f32_parts(a, A, ea);
  f32_parts(b, B, eb);
  f32_parts(c, C, ec);
  // candidate in units of 2^-25: r32 in [1, 4)
  uint32_t rb;
  memcpy(&rb, &r32, 4);
  const uint32_t R = (rb & 0x7fffffu) | 0x800000u;
  const int er = (int)(rb >> 23) - 127;  // 0 or 1
  const uint64_t step = er == 0 ? 4ull : 8ull;  // one ulp of r32 in units of 2^-25
  const uint64_t Mr = (uint64_t)R * step;
  const bool pow2 = (rb & 0x7fffffu) == 0u;
  const uint64_t Mlo = Mr - (pow2 ? step / 4 : step / 2);  // midpoint below
  const uint64_t Mhi = Mr + step / 2;                      // midpoint above
  const int slo = sign_s_minus_m2(A, B, eb, C, ec, Mlo);
  uint32_t out = rb;
  if (slo < 0 || (slo == 0 && (rb & 1u))) {
    out = rb - 1u;  // below the lower midpoint (or a tie that goes to the even lower value)
  } else if (slo > 0) {
    const int shi = sign_s_minus_m2(A, B, eb, C, ec, Mhi);
    if (shi > 0 || (shi == 0 && (rb & 1u))) out = rb + 1u;
  }
  float f;
  memcpy(&f, &out, 4);
  return f;
}

}  // namespace exact
}  // namespace ivc
