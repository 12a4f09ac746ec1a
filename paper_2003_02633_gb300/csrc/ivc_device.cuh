// Device arithmetic of inline 3-vector compression (Trojak & Witherden,
// arXiv:2003.02633) for sm_103a.
//
// Every rounding decision the method makes is taken in FP32 arithmetic with a
// stated error bound; the rare inputs whose decision the bound does not
// settle are decided again in 64/128-bit integer arithmetic (ivc_exact.cuh,
// noinline helpers, off the common path).  No floating point wider than FP32.
//
// Encoding (Sec. 2.1, 2.3, 3).
//   magnitude: RN32(|x|) from a float-float sum of squares and a
//     float-float square root (error < 2^-44); within 2^-42 of an FP32
//     rounding midpoint the exact sign of |x|^2 - m^2 at the midpoint m
//     decides.  Exponent rebiased, mantissa truncated (Sec. 2.3).
//   angles: n = nint(t) (Eq. a_disc).  An FP32 estimate of t, good to a few
//     hundredths of a bin, names the one rounding boundary k + 1/2 that can
//     matter; a side-of-boundary test of the input against that boundary's
//     direction decides k or k + 1:
//       theta: sign(y cos(theta_h) - x sin(theta_h)),
//       phi:   sign(rho cos(phi_h) - z sin(phi_h)),  rho = sqrt(x^2 + y^2),
//     with cos/sin of the boundary in float-float (about 2^-42 relative) and
//     error-free products; |test| below 2^-40 of its terms -> the test again
//     with cos/sin to about 2^-57 (integer Taylor series).
//     Exact ties (theta = 0, phi = pi/2) give a test value of exactly zero and
//     round up.
//
// Decoding (Eq. a_inv, Eq. cart2sphere).  theta^ = pi (2 n_theta - N) / N and
// phi^ = pi (2 n_phi) / (2M) are rational multiples of pi.  Each angle pi m / D
// is folded exactly, in integers, onto [0, pi/4]; cos and sin there come from
// a shared-memory table of float-float values at multiples of 2^s units
// (pi / (2D) each; at most 1024 entries) plus a Taylor step for the signed
// remainder.
// The products r cos(theta) sin(phi) etc. are formed in float-float and
// rounded away from zero with a directed-rounding FMA; when the value lies
// within 2^-40 (relative) of an FP32 grid point the vector is decoded again
// with cos/sin and products to about 2^-56 (integer arithmetic).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "ivc_exact.cuh"

namespace ivc {

enum : int { MAP_UNIFORM = 0, MAP_TANH = 1, MAP_FRACSPLIT = 2 };

// Relative error bounds of the FP32 paths (see the design notes for the
// derivation); the ambiguity thresholds include a safety factor.
constexpr float kDecodeAmbig = 9.094947e-13f;   // 2^-40
constexpr float kSideAmbig = 9.094947e-13f;     // 2^-40
constexpr float kNormAmbig = 2.2737368e-13f;    // 2^-42

// cos/sin of one table angle, each as head + tail.
struct __align__(16) TabEntry {
  float ch, cl, sh, sl;
};

struct FF {
  float h, l;
};

// Everything a kernel needs to know about a format (built on the host).
struct DevFormat {
  uint32_t sh_phi, sh_m, sh_e;      // field shifts
  uint32_t mask_e, mask_m;          // field masks (low bits)
  uint32_t mask_phi, mask_theta;
  uint32_t m_shift;                 // 23 - man_bits
  uint64_t mask_np;                 // fractional split: p + t low bits
  int32_t e_off;                    // exponent field = E8 + e_off
  int32_t e_maxn;                   // largest normal exponent field, 2^e - 2
  int32_t e_all;                    // 2^e - 1 (non-finite)
  int32_t N, M;                     // n_theta_max, n_phi_max
  int32_t under_mode, over_mode;
  float tscale_t, thalf_t, tmax_t;  // t_theta = thalf + theta * tscale, clamp
  float tscale_p, tmax_p;           // t_phi = phi * tscale
  // uniform / fractional split: folded sin/cos tables (theta then phi)
  int32_t Dt, Dp;                   // theta grid pi m / N, phi grid pi m / (2M)
  int32_t nent_t, nent_p;           // table entries
  int32_t st, sp;                   // table step 2^s units
  float Kt_h, Kt_l, Kp_h, Kp_l;     // pi / (2 D) in float-float
  uint64_t Kxt_m, Kxp_m;            // pi / (2 D) = Kx_m 2^Kx_e (64-bit, exact paths)
  int32_t Kxt_e, Kxp_e;
  const TabEntry *tab;              // global, nent_t + nent_p entries
  // uniform / fractional split: cos, sin of phi^_k = pi k / M for k = 0 ..
  // floor(M / 2), one entry per code of the lower half of the phi range
  // (global; read by the fast decoders; null where a caller has no table)
  const TabEntry *phi_tab;
  uint64_t div_magic;               // ceil(2^64 / (N + 1)) for the split
  // tanh companding
  float gam, tanh_c, tanh_inv2c;    // gamma, c = tanh(gamma), 1 / (2c)
  const TabEntry *dec_t, *dec_p;    // cos/sin of theta^_n (N+1), phi^_n (M+1)
  const TabEntry *bnd_t, *bnd_p;    // cos/sin at boundaries k + 1/2 (N, M)
  // tanh companding, fast encoder: bin coordinate t at nodes j pi / 1024 of
  // |theta| in [0, pi] (nest_t entries) and of phi in [0, pi/2] (nest_p):
  // (floor t, t - floor t, dt/dangle, d2t/dangle2 / 2) per node
  const TabEntry *est_tab;
  int32_t nest_t, nest_p;
};

// --------------------------------------------------------------------------
// Exact integer folding of pi m / D onto [0, pi/4].

struct Fold {
  int b;       // folded angle pi b / (2D), b in [0, D/2]
  bool swap;   // cos and sin exchange
  bool cneg;   // cos negative
  bool sneg;   // sin negative
};

__device__ __forceinline__ Fold fold_grid(int m, int D) {
  Fold f;
  f.sneg = m < 0;
  const int a = abs(m);
  f.cneg = 2 * a > D;
  const int a1 = f.cneg ? D - a : a;   // pi a1 / D in [0, pi/2]
  f.swap = 4 * a1 > D;
  f.b = f.swap ? D - 2 * a1 : 2 * a1;  // pi b / (2D) in [0, pi/4]
  return f;
}

// cos and sin (both >= 0) of pi b / (2D) from the head table (entries at
// b = h 2^s) and a Taylor step over the signed remainder l = b - h 2^s,
// |l| <= 2^(s-1) (h = b / 2^s rounded to nearest): relative error below 2^-42.
// Fast2Sum preconditions: |cA| >= |sA beta| always; |sA| >= |cA beta| when
// h >= 1 (tan A >= A >= |beta|), and sA = 0 when h = 0 (then l >= 0).
__device__ __forceinline__ void sincos_folded(int b, const TabEntry *__restrict__ tab, int s,
                                              float Kh, float Kl, FF &c, FF &sn) {
  const int h = (s > 0) ? ((b + (1 << (s - 1))) >> s) : b;
  const float lf = (float)(b - (h << s));
  const TabEntry e = tab[h];
  // beta = l pi / (2D) in float-float
  const float bh = lf * Kh;
  const float bl = fmaf(lf, Kh, -bh) + lf * Kl;
  const float b2 = bh * bh;
  const float u = b2 * fmaf(b2, -1.0f / 24.0f, 0.5f);                     // 1 - cos(beta)
  const float stail = fmaf(bh * b2, fmaf(b2, 1.0f / 120.0f, -1.0f / 6.0f), bl);  // sin(beta) - bh
  // cos(A + beta) = cA - cA u - sA sin(beta)
  const float P = e.sh * bh;
  const float Pe = fmaf(e.sh, bh, -P);
  const float Ch = e.ch - P;
  const float Ce = (e.ch - Ch) - P;
  float Cl = Ce + e.cl;
  Cl = Cl - Pe;
  Cl = fmaf(-e.ch, u, Cl);
  Cl = fmaf(-e.sh, stail, Cl);
  Cl = fmaf(-e.sl, bh, Cl);
  // sin(A + beta) = sA - sA u + cA sin(beta)
  const float Q = e.ch * bh;
  const float Qe = fmaf(e.ch, bh, -Q);
  const float Sh = e.sh + Q;
  const float Se = Q - (Sh - e.sh);
  float Sl = Se + Qe;
  Sl = Sl + e.sl;
  Sl = fmaf(-e.sh, u, Sl);
  Sl = fmaf(e.ch, stail, Sl);
  Sl = fmaf(e.cl, bh, Sl);
  c.h = Ch; c.l = Cl;
  sn.h = Sh; sn.l = Sl;
}

// cos and sin of pi m / D (m in [-D, D]): magnitudes and signs.
__device__ __forceinline__ void sincospi_grid(int m, int D, const TabEntry *__restrict__ tab,
                                              int s, float Kh, float Kl, FF &c, FF &sn,
                                              bool &cneg, bool &sneg) {
  const Fold f = fold_grid(m, D);
  cneg = f.cneg;
  sneg = f.sneg;
  FF cc, ss;
  sincos_folded(f.b, tab, s, Kh, Kl, cc, ss);
  c = f.swap ? ss : cc;
  sn = f.swap ? cc : ss;
}

__device__ __forceinline__ FF neg_if(FF v, bool n) {
  return n ? FF{-v.h, -v.l} : v;
}

// Side test a c - b s for exact FP32 a (+ tail a_l), b and float-float c, s.
// Returns +1 / 0 (for "< 0") when settled, -1 when |value| is within the
// error bound.
__device__ __forceinline__ int side_ge(float a, float a_l, FF c, float b, FF s) {
  const float p1 = a * c.h;
  const float e1 = fmaf(a, c.h, -p1);
  const float p2 = b * s.h;
  const float e2 = fmaf(b, s.h, -p2);
  float lo = e1 - e2;
  lo = fmaf(a, c.l, lo);
  lo = fmaf(-b, s.l, lo);
  lo = fmaf(a_l, c.h, lo);
  const float d = (p1 - p2) + lo;
  const float bound = kSideAmbig * (fabsf(p1) + fabsf(p2));
  if (fabsf(d) <= bound && d != 0.0f) return -1;
  if (d == 0.0f && bound != 0.0f && (p1 != p2 || lo != 0.0f)) return -1;
  return d >= 0.0f ? 1 : 0;
}

// Round-up of r * (a * b) for non-negative float-floats a, b; sets amb when
// the value lies within the decode error bound of an FP32 grid point.
__device__ __forceinline__ float ru_prod3(float r, FF a, FF b, bool &amb) {
  const float P = a.h * b.h;
  const float Pe = fmaf(a.h, b.h, -P);
  const float Pl = fmaf(a.h, b.l, fmaf(a.l, b.h, Pe));
  const float t = r * Pl;
  const float d = kDecodeAmbig * (r * P);
  const float x0 = __fmaf_ru(r, P, t - d);
  const float x1 = __fmaf_ru(r, P, t + d);
  amb |= (x0 != x1);
  return x1;
}

__device__ __forceinline__ float ru_prod2(float r, FF a, bool &amb) {
  const float t = r * a.l;
  const float d = kDecodeAmbig * (r * a.h);
  const float x0 = __fmaf_ru(r, a.h, t - d);
  const float x1 = __fmaf_ru(r, a.h, t + d);
  amb |= (x0 != x1);
  return x1;
}

__device__ __forceinline__ float apply_sign(float mag, bool neg) {
  return (neg && mag != 0.0f) ? -mag : mag;
}

// --------------------------------------------------------------------------
// Field access.

template <int MAP>
__device__ __forceinline__ void unpack_angles(uint64_t w, const DevFormat &F, int &nt, int &np) {
  if (MAP == MAP_FRACSPLIT) {
    const uint64_t npk = w & F.mask_np;
    const uint64_t q = __umul64hi(npk, F.div_magic);  // floor(npk / (N + 1)), npk < 2^40
    nt = (int)(npk - q * (uint64_t)(F.N + 1));
    // n_p beyond (n_phi_max + 1)(n_theta_max + 1) - 1 is not a valid code: clamp
    // n_phi so that every table index stays in range.
    np = q > (uint64_t)F.M ? F.M : (int)q;
  } else {
    np = (int)((uint32_t)(w >> F.sh_phi) & F.mask_phi);
    nt = (int)((uint32_t)w & F.mask_theta);
  }
}

template <int MAP>
__device__ __forceinline__ uint64_t pack_angles(int nt, int np, const DevFormat &F) {
  if (MAP == MAP_FRACSPLIT) return (uint64_t)np * (uint64_t)(F.N + 1) + (uint64_t)nt;
  return ((uint64_t)np << F.sh_phi) | (uint64_t)nt;
}

__device__ __forceinline__ float magnitude_of(uint32_t E, uint32_t mant, const DevFormat &F) {
  const uint32_t rbits = ((uint32_t)((int)E - F.e_off) << 23) | (mant << F.m_shift);
  return (E == 0u) ? 0.0f : __uint_as_float(rbits);
}

// --------------------------------------------------------------------------
// Decode one word (Eq. a_inv, Eq. cart2sphere).

// Exact-path decode of a finite word (the fallback of decode_word): cos/sin
// and the products to about 2^-56 in integer arithmetic, rounded away from
// zero.
template <int MAP>
static __device__ __noinline__ float3 decode_word_exact(uint64_t w, const DevFormat &F) {
  using namespace exact;
  const uint32_t E = (uint32_t)(w >> F.sh_e) & F.mask_e;
  const uint32_t mant = (uint32_t)(w >> F.sh_m) & F.mask_m;
  int nt, np;
  unpack_angles<MAP>(w, F, nt, np);
  SF ct, st, cp, sp;
  bool ctn, stn, cpn, spn;
  if (MAP == MAP_TANH) {
    const TabEntry et = F.dec_t[nt];
    const TabEntry ep = F.dec_p[np];
    ct = sf_from_ff(et.ch, et.cl, ctn);
    st = sf_from_ff(et.sh, et.sl, stn);
    cp = sf_from_ff(ep.ch, ep.cl, cpn);
    sp = sf_from_ff(ep.sh, ep.sl, spn);
  } else {
    sincospi_grid(2 * nt - F.N, F.Dt, SF{F.Kxt_m, F.Kxt_e, false}, ct, st, ctn, stn);
    sincospi_grid(2 * np, F.Dp, SF{F.Kxp_m, F.Kxp_e, false}, cp, sp, cpn, spn);
  }
  const SF r = sf_from_float(magnitude_of(E, mant, F));
  const SF R = sf_mul(r, sp);
  return make_float3(apply_sign(ra32(sf_mul(R, ct)), ctn), apply_sign(ra32(sf_mul(R, st)), stn),
                     apply_sign(ra32(sf_mul(r, cp)), cpn));
}

// EXACT: every finite word through decode_word_exact (validation entry points).
template <int MAP, bool EXACT = false>
__device__ __forceinline__ float3 decode_word(uint64_t w, const DevFormat &F,
                                              const TabEntry *__restrict__ tab_t,
                                              const TabEntry *__restrict__ tab_p) {
  const uint32_t E = (uint32_t)(w >> F.sh_e) & F.mask_e;
  const uint32_t mant = (uint32_t)(w >> F.sh_m) & F.mask_m;
  int nt, np;
  unpack_angles<MAP>(w, F, nt, np);
  FF ct, st, cp, sp;
  bool ctn, stn, cpn, spn;
  if (MAP == MAP_TANH) {
    const TabEntry et = F.dec_t[nt];
    const TabEntry ep = F.dec_p[np];
    ctn = et.ch < 0.0f; stn = et.sh < 0.0f; cpn = ep.ch < 0.0f; spn = false;
    ct = neg_if(FF{et.ch, et.cl}, ctn);
    st = neg_if(FF{et.sh, et.sl}, stn);
    cp = neg_if(FF{ep.ch, ep.cl}, cpn);
    sp = FF{ep.sh, ep.sl};
  } else {
    sincospi_grid(2 * nt - F.N, F.Dt, tab_t, F.st, F.Kt_h, F.Kt_l, ct, st, ctn, stn);
    sincospi_grid(2 * np, F.Dp, tab_p, F.sp, F.Kp_h, F.Kp_l, cp, sp, cpn, spn);
  }
  if (E == (uint32_t)F.e_all) {
    const float nan = __int_as_float(0x7fc00000);
    if (mant != 0u) return make_float3(nan, nan, nan);
    const float inf = __int_as_float(0x7f800000);  // infinite magnitude
    const float x = (ct.h != 0.0f && sp.h != 0.0f) ? inf : 0.0f;
    const float y = (st.h != 0.0f && sp.h != 0.0f) ? inf : 0.0f;
    const float z = (cp.h != 0.0f) ? inf : 0.0f;
    return make_float3(apply_sign(x, ctn), apply_sign(y, stn), apply_sign(z, cpn));
  }
  if (EXACT) return decode_word_exact<MAP>(w, F);
  const float r = magnitude_of(E, mant, F);
  bool amb = false;
  const float x = ru_prod3(r, ct, sp, amb);
  const float y = ru_prod3(r, st, sp, amb);
  const float z = ru_prod2(r, cp, amb);
  if (amb) return decode_word_exact<MAP>(w, F);
  return make_float3(apply_sign(x, ctn), apply_sign(y, stn), apply_sign(z, cpn));
}

// --------------------------------------------------------------------------
// Encode one vector (Sec. 2.1, 2.3, 3).  flags: bit 0 overflow, bit 1
// underflow, bit 2 NaN.

__device__ __forceinline__ float pow2f(int e) {  // 2^e for e in [-126, 127]
  return __uint_as_float((uint32_t)(e + 127) << 23);
}

// RN32 of the norm of the scaled vector, decided exactly (the fallback of the
// float-float norm; r32 is its candidate).
static __device__ __noinline__ float norm_rn_exact(float xs, float ys, float zs, float r32) {
  return exact::norm_rn(xs, ys, zs, r32);
}

// Exact-path side tests (the fallbacks of side_ge): 1 when the input lies on
// or above boundary k + 1/2, else 0.
// theta: sign(y cos(t_b) - x sin(t_b)) >= 0.
template <int MAP>
static __device__ __noinline__ int side_theta_exact(float xs, float ys, int k, const DevFormat &F) {
  using namespace exact;
  SF c, s;
  bool cn, sn;
  if (MAP == MAP_TANH) {
    const TabEntry e = F.bnd_t[k];
    c = sf_from_ff(e.ch, e.cl, cn);
    s = sf_from_ff(e.sh, e.sl, sn);
  } else {
    sincospi_grid(2 * k + 1 - F.N, F.Dt, SF{F.Kxt_m, F.Kxt_e, false}, c, s, cn, sn);
  }
  const SF A = sf_mul(sf_from_float(ys), c);
  const SF B = sf_mul(sf_from_float(xs), s);
  return side_of(A, signbit(ys) != cn, B, signbit(xs) != sn);
}

// phi: sign(rho cos(p_b) - z sin(p_b)) >= 0 with rho = sqrt(x^2 + y^2) >= 0;
// the magnitudes rho |cos| and |z| sin are compared through their squares.
template <int MAP>
static __device__ __noinline__ int side_phi_exact(float xs, float ys, float zs, int k,
                                                  const DevFormat &F) {
  using namespace exact;
  SF c, s;
  bool cn, sn;
  if (MAP == MAP_TANH) {
    const TabEntry e = F.bnd_p[k];
    c = sf_from_ff(e.ch, e.cl, cn);
    s = sf_from_ff(e.sh, e.sl, sn);
  } else {
    sincospi_grid(2 * k + 1, F.Dp, SF{F.Kxp_m, F.Kxp_e, false}, c, s, cn, sn);
  }
  const SF X = sf_from_float(xs), Y = sf_from_float(ys), Z = sf_from_float(zs);
  const SF rho2 = sf_add(sf_mul(X, X), sf_mul(Y, Y));
  const SF A2 = sf_mul(rho2, sf_mul(c, c));
  const SF B2 = sf_mul(sf_mul(Z, Z), sf_mul(s, s));
  return side_of(A2, cn, B2, signbit(zs) != sn);
}

// EXACT: every decision through the exact helpers (validation entry points).
template <int MAP, bool EXACT = false>
__device__ __forceinline__ uint64_t encode_vec(float x, float y, float z, const DevFormat &F,
                                               const TabEntry *__restrict__ tab_t,
                                               const TabEntry *__restrict__ tab_p,
                                               uint32_t &flags) {
  if (isnan(x) || isnan(y) || isnan(z)) {
    flags |= 4u;
    return ((uint64_t)F.e_all << F.sh_e) | (1ull << F.sh_m);
  }
  float amax = fmaxf(fabsf(x), fmaxf(fabsf(y), fabsf(z)));
  if (amax == 0.0f) return 0ull;
  const bool inf_in = isinf(amax);
  if (inf_in) {
    x = isinf(x) ? copysignf(1.0f, x) : copysignf(0.0f, x);
    y = isinf(y) ? copysignf(1.0f, y) : copysignf(0.0f, y);
    z = isinf(z) ? copysignf(1.0f, z) : copysignf(0.0f, z);
    amax = 1.0f;
  }
  // Exact power-of-two scaling to max component in [1, 2).
  int S;
  {
    const uint32_t ub = __float_as_uint(amax);
    const int ex = (int)(ub >> 23);
    S = (ex != 0) ? 127 - ex : 118 + __clz((int)(ub & 0x7fffffu));
  }
  float xs, ys, zs;
  if (S >= -126 && S <= 127) {
    const float sc = pow2f(S);
    xs = x * sc; ys = y * sc; zs = z * sc;
  } else {
    const int S1 = S / 2, S2 = S - S / 2;
    const float s1 = pow2f(S1), s2 = pow2f(S2);
    xs = (x * s1) * s2; ys = (y * s1) * s2; zs = (z * s1) * s2;
  }
  // Sum of squares in float-float.
  const float px = xs * xs, ex_ = fmaf(xs, xs, -px);
  const float py = ys * ys, ey = fmaf(ys, ys, -py);
  const float pz = zs * zs, ez = fmaf(zs, zs, -pz);
  float r2h = px + py;
  float t = r2h - px;
  const float r2l = ((px - (r2h - t)) + (py - t)) + (ex_ + ey);
  float sh = r2h + pz;
  t = sh - r2h;
  const float sl = ((r2h - (sh - t)) + (pz - t)) + (r2l + ez);
  // Float-float square root and RN32 of it.
  const float y0 = rsqrtf(sh);
  const float hy0 = 0.5f * y0;
  const float r0 = sh * y0;
  const float rh = fmaf(fmaf(-r0, r0, sh) + sl, hy0, r0);
  const float rl = (fmaf(-rh, rh, sh) + sl) * hy0;
  float r32 = rh + rl;
  {
    // distance of rh + rl from the FP32 rounding midpoints around r32
    const float half_ulp = __uint_as_float((__float_as_uint(r32) & 0x7f800000u) - (24u << 23));
    const float dev = fabsf((rh - r32) + rl);
    // a power of two has its lower midpoint a quarter ulp away: re-check those too
    if (EXACT || half_ulp - dev <= kNormAmbig * r32 || (__float_as_uint(r32) & 0x7fffffu) == 0u)
      r32 = norm_rn_exact(xs, ys, zs, r32);
  }
  const uint32_t rb = __float_as_uint(r32);
  const int E8 = (int)(rb >> 23) - S;
  int Ef = E8 + F.e_off;
  uint32_t mant = (rb & 0x7fffffu) >> F.m_shift;
  const bool over = inf_in || E8 > 254 || Ef > F.e_maxn;
  const bool under = !over && (E8 < 1 || Ef < 1);

  // theta: estimate, then one side test.
  int nt, np;
  {
    float tt;
    if (MAP == MAP_TANH) {
      const float psi = fmaf(atan2f(ys, xs), 0.15915494309189535f, 0.5f);
      tt = (tanhf(F.gam * fmaf(2.0f, psi, -1.0f)) + F.tanh_c) * F.tanh_inv2c * (float)F.N;
    } else {
      tt = fmaf(atan2f(ys, xs), F.tscale_t, F.thalf_t);
    }
    tt = fminf(fmaxf(tt, 0.0f), F.tmax_t);
    const int k = (int)tt;
    FF c, s;
    if (MAP == MAP_TANH) {
      const TabEntry e = F.bnd_t[k];
      c = FF{e.ch, e.cl};
      s = FF{e.sh, e.sl};
    } else {
      bool cn, sn;
      sincospi_grid(2 * k + 1 - F.N, F.Dt, tab_t, F.st, F.Kt_h, F.Kt_l, c, s, cn, sn);
      c = neg_if(c, cn);
      s = neg_if(s, sn);
    }
    int side = EXACT ? -1 : side_ge(ys, 0.0f, c, xs, s);
    if (side < 0) side = side_theta_exact<MAP>(xs, ys, k, F);
    nt = k + side;
  }
  // phi: rho = sqrt(x^2 + y^2) in float-float.
  {
    float rho_h = 0.0f, rho_l = 0.0f;
    if (r2h > 0.0f) {
      const float y1 = rsqrtf(r2h);
      const float hy1 = 0.5f * y1;
      const float q0 = r2h * y1;
      rho_h = fmaf(fmaf(-q0, q0, r2h) + r2l, hy1, q0);
      rho_l = (fmaf(-rho_h, rho_h, r2h) + r2l) * hy1;
    }
    float tp;
    if (MAP == MAP_TANH) {
      const float psi = atan2f(rho_h, zs) * 0.3183098861837907f;
      tp = (tanhf(F.gam * fmaf(2.0f, psi, -1.0f)) + F.tanh_c) * F.tanh_inv2c * (float)F.M;
    } else {
      tp = atan2f(rho_h, zs) * F.tscale_p;
    }
    tp = fminf(fmaxf(tp, 0.0f), F.tmax_p);
    const int k = (int)tp;
    FF c, s;
    if (MAP == MAP_TANH) {
      const TabEntry e = F.bnd_p[k];
      c = FF{e.ch, e.cl};
      s = FF{e.sh, e.sl};
    } else {
      bool cn, sn;
      sincospi_grid(2 * k + 1, F.Dp, tab_p, F.sp, F.Kp_h, F.Kp_l, c, s, cn, sn);
      c = neg_if(c, cn);
    }
    int side = EXACT ? -1 : side_ge(rho_h, rho_l, c, zs, s);
    if (side < 0) side = side_phi_exact<MAP>(xs, ys, zs, k, F);
    np = k + side;
  }
  if (nt == F.N) nt = 0;
  if (np == 0 || np == F.M) nt = 0;

  if (under) {
    flags |= 2u;
    if (F.under_mode == 1) return 0ull;
    Ef = 1;
    mant = 0u;
  }
  if (over) {
    flags |= 1u;
    if (F.over_mode == 1) {
      Ef = F.e_all;
      mant = 0u;
    } else {
      Ef = F.e_maxn;
      mant = F.mask_m;
    }
  }
  return ((uint64_t)(uint32_t)Ef << F.sh_e) | ((uint64_t)mant << F.sh_m) |
         pack_angles<MAP>(nt, np, F);
}

// --------------------------------------------------------------------------
// Shared-memory table staging for the uniform grids.

template <int MAP>
__device__ __forceinline__ void stage_tables(const DevFormat &F, TabEntry *smem) {
  if (MAP == MAP_TANH) return;
  const int total = F.nent_t + F.nent_p;
  const float4 *src = reinterpret_cast<const float4 *>(F.tab);
  float4 *dst = reinterpret_cast<float4 *>(smem);
  for (int i = threadIdx.x; i < total; i += blockDim.x) dst[i] = __ldg(src + i);
  __syncthreads();
}

}  // namespace ivc
