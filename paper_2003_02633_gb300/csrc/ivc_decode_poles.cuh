// Pair decodes built on the fast path: with the poles of the sphere settled in
// place (decode2_poles), and in plain FP32 for consumers that need the
// components only to within a few ulps (decode2_f32).
//
// At n_phi = 0 or n_phi_max the decoded vector is exactly (0, 0, +r^) or
// (0, 0, -r^): sin(phi^) = 0 and cos(phi^) = +-1 make every product exact
// (Sec. 2.2, Eq. a_inv), whatever n_theta holds.  The directed-rounding test
// of the fast decoder cannot tell an exact product from one that only lies
// close to an FP32 number, so it flags these words, and a flux with a
// vanishing velocity component (the Taylor-Green initial state: the row
// rho w u + p e_z = (0, 0, p)) would send one row in five to the generic
// decoder.  Other flagged words (ambiguous roundings, non-finite words) still
// go there.
#pragma once

#include "ivc_fast.cuh"

namespace ivc {
namespace fast {

template <class G>
__device__ __forceinline__ void pole_or_generic(uint64_t w, const DevFormat &F,
                                                const TabEntry *tab_t, const TabEntry *tab_p,
                                                float &x, float &y, float &z) {
  const uint32_t hi = (uint32_t)(w >> 32), lo = (uint32_t)w;
  uint32_t nt, np;
  G::unpack(hi, lo, nt, np);
  const uint32_t E = G::efield(hi);
  if (E != 0u && E != G::EALL && (np == 0u || np == (uint32_t)G::M)) {
    const float r = G::mag(hi);
    x = 0.0f;
    y = 0.0f;
    z = np == 0u ? r : -r;
    return;
  }
  const float3 v = decode_generic<G::MAP>(w, F, tab_t, tab_p);
  x = v.x;
  y = v.y;
  z = v.z;
}

template <class G>
__device__ __forceinline__ void decode2_poles(uint64_t w0, uint64_t w1, const DevFormat &F,
                                              const TabEntry *tab_t, const TabEntry *tab_p,
                                              float2 &X, float2 &Y, float2 &Z) {
  bool s0, s1;
  decode2<G, true>(w0, w1, F, tab_t, tab_p, X, Y, Z, s0, s1);
  if (s0) pole_or_generic<G>(w0, F, tab_t, tab_p, X.x, Y.x, Z.x);
  if (s1) pole_or_generic<G>(w1, F, tab_t, tab_p, X.y, Y.y, Z.y);
}

// cos and sin of pi b / (2D) (b the folded code, |angle| <= pi/4) in plain
// FP32 for both elements: the heads of the shared table entry at the nearest
// multiple of 2^S and the Taylor terms 1 - beta^2/2 and beta - beta^3/6 of the
// remainder beta (|beta| <= 7.7e-4, so the next terms are below 2^-45).
// Relative error of the cosine at most 3 2^-24 and of the sine at most
// 10 2^-24: the table heads carry 2^-24 each, beta 2 2^-24, the Taylor terms
// and the last FMA a few 2^-24 more, and for a negative beta the remainder's
// term cancels at most half of the head's sine (head angle >= the table step
// >= 2 |beta|; at the first entry, head angle 0, beta >= 0).
template <int S>
__device__ __forceinline__ void sincos2_f32(float2 b, const TabEntry *__restrict__ tab, float Kh,
                                            float2 &c, float2 &s) {
  const float2 hb = fma2(b, bc(1.0f / (float)(1 << S)), bc(kMagic));
  const float2 hf = add2(hb, bc(-kMagic));
  const float2 lf = fma2(hf, bc(-(float)(1 << S)), b);
  const TabEntry e0 = tab[__float_as_uint(hb.x) - kMagicBits];
  const TabEntry e1 = tab[__float_as_uint(hb.y) - kMagicBits];
  const float2 X = make_float2(e0.ch, e1.ch), Y = make_float2(e0.sh, e1.sh);
  const float2 bh = mul2(lf, bc(Kh));
  const float2 b2 = mul2(bh, bh);
  const float2 cd = fma2(b2, bc(-0.5f), bc(1.0f));
  const float2 sd = fma2(mul2(bh, b2), bc(-1.0f / 6.0f), bh);
  c = fma2(X, cd, neg2(mul2(Y, sd)));
  s = fma2(Y, cd, mul2(X, sd));
}

// Pair decode in plain FP32 for consumers that need each component only to
// within a few units in the last place (the FP32 contractions of Algorithm 1
// and of the FR steps).  Both angles are folded onto [0, pi/4] and evaluated
// by sincos2_f32 from the shared-memory head tables (no global-memory gather,
// so nothing waits on L2 when the codes of neighbouring words scatter), and the
// products r^ sin(phi^) cos(theta^), r^ sin(phi^) sin(theta^), r^ cos(phi^)
// are rounded twice at most.  Relative error per component at most 22 2^-24
// (10 2^-24 for each angle's cosine or sine, 2^-24 per product rounding), a
// few 2^-24 in practice; exact at the poles and for zero words; non-finite
// words take the generic decoder.
template <class G>
__device__ __forceinline__ void decode2_f32(uint64_t w0, uint64_t w1, const DevFormat &F,
                                            const TabEntry *tab_t, const TabEntry *tab_p,
                                            float2 &X, float2 &Y, float2 &Z) {
  const uint32_t hi0 = (uint32_t)(w0 >> 32), lo0 = (uint32_t)w0;
  const uint32_t hi1 = (uint32_t)(w1 >> 32), lo1 = (uint32_t)w1;
  const uint32_t E0 = G::efield(hi0), E1 = G::efield(hi1);
  const float2 r = make_float2(E0 == 0u ? 0.0f : G::mag(hi0), E1 == 0u ? 0.0f : G::mag(hi1));
  uint32_t nt0, np0, nt1, np1;
  G::unpack(hi0, lo0, nt0, np0);
  G::unpack(hi1, lo1, nt1, np1);
  // phi^ = pi (2 n_phi) / (2M); sin(phi^) >= 0, cos(phi^) < 0 past pi/2
  const float2 npf = add2(make_float2(__uint_as_float(np0 | 0x4B000000u),
                                      __uint_as_float(np1 | 0x4B000000u)),
                          bc(-8388608.0f));
  const Fold2 fp = fold2(add2(npf, npf), (float)(2 * G::M));
  float2 pc, ps;
  sincos2_f32<G::SP>(fp.b, tab_p, F.Kp_h, pc, ps);
  const float2 cph = sel2(fp.swap0, fp.swap1, ps, pc);
  const float2 sph = sel2(fp.swap0, fp.swap1, pc, ps);
  // theta^ = pi (2 n_theta - N) / N
  const float2 ntf = add2(make_float2(__uint_as_float(nt0 | 0x4B000000u),
                                      __uint_as_float(nt1 | 0x4B000000u)),
                          bc(-8388608.0f));
  const float2 mt = fma2(ntf, bc(2.0f), bc(-(float)G::N));
  const Fold2 ft = fold2(make_float2(fabsf(mt.x), fabsf(mt.y)), (float)G::N);
  float2 cc, ss;
  sincos2_f32<G::ST>(ft.b, tab_t, F.Kt_h, cc, ss);
  const float2 ct = sel2(ft.swap0, ft.swap1, ss, cc);
  const float2 st = sel2(ft.swap0, ft.swap1, cc, ss);
  const float2 R = mul2(r, sph);  // r^ sin(phi^)
  // + 0: a zero component is +0, as in the canonical decode
  X = fma2(R, make_float2(ft.cneg0 ? -ct.x : ct.x, ft.cneg1 ? -ct.y : ct.y), bc(0.0f));
  Y = fma2(R, make_float2(copysignf(st.x, mt.x), copysignf(st.y, mt.y)), bc(0.0f));
  Z = fma2(r, make_float2(fp.cneg0 ? -cph.x : cph.x, fp.cneg1 ? -cph.y : cph.y), bc(0.0f));
  if (E0 == G::EALL) {
    const float3 v = decode_generic<G::MAP>(w0, F, tab_t, tab_p);
    X.x = v.x; Y.x = v.y; Z.x = v.z;
  }
  if (E1 == G::EALL) {
    const float3 v = decode_generic<G::MAP>(w1, F, tab_t, tab_p);
    X.y = v.x; Y.y = v.y; Z.y = v.z;
  }
}

}  // namespace fast
}  // namespace ivc
