// Pair decodes built on the fast path: with the poles of the sphere settled in
// place (decode2_poles), and rounded to nearest for consumers that need the
// components only to within an ulp (decode2_near).
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

}  // namespace fast
}  // namespace ivc

namespace ivc {
namespace fast {

// Pair decode for a consumer that only needs the decoded components to within
// one unit in the last place (the FP32 products of Algorithm 1): the same
// float-float evaluation of r^ cos(theta^) sin(phi^) ... as decode2, rounded
// to nearest instead of away from zero, so it needs no ambiguity test and no
// generic fallback except for non-finite words.  Within 1.5 units of the
// last place of the canonical decoded value.
template <class G>
__device__ __forceinline__ void decode2_near(uint64_t w0, uint64_t w1, const DevFormat &F,
                                             const TabEntry *tab_t, const TabEntry *tab_p,
                                             float2 &X, float2 &Y, float2 &Z) {
  const uint32_t hi0 = (uint32_t)(w0 >> 32), lo0 = (uint32_t)w0;
  const uint32_t hi1 = (uint32_t)(w1 >> 32), lo1 = (uint32_t)w1;
  const uint32_t E0 = G::efield(hi0), E1 = G::efield(hi1);
  const float r0 = E0 == 0u ? 0.0f : G::mag(hi0);
  const float r1 = E1 == 0u ? 0.0f : G::mag(hi1);
  uint32_t nt0, np0, nt1, np1;
  G::unpack(hi0, lo0, nt0, np0);
  G::unpack(hi1, lo1, nt1, np1);
  const float2 ntf = add2(make_float2(__uint_as_float(nt0 | 0x4B000000u),
                                      __uint_as_float(nt1 | 0x4B000000u)),
                          bc(-8388608.0f));
  FF2 cp, sp;
  bool pneg0, pneg1;
  phi_pair<G, true>(np0, np1, F, tab_p, cp, sp, pneg0, pneg1);
  const float2 mt = fma2(ntf, bc(2.0f), bc(-(float)G::N));
  const Fold2 ft = fold2(make_float2(fabsf(mt.x), fabsf(mt.y)), (float)G::N);
  FF2 cc, ss;
  sincos2<G::ST>(ft.b, tab_t, F.Kt_h, F.Kt_l, cc, ss);
  FF2 ct, st;
  ct.h = sel2(ft.swap0, ft.swap1, ss.h, cc.h);
  ct.l = sel2(ft.swap0, ft.swap1, ss.l, cc.l);
  st.h = sel2(ft.swap0, ft.swap1, cc.h, ss.h);
  st.l = sel2(ft.swap0, ft.swap1, cc.l, ss.l);
  const float2 r = make_float2(r0, r1);
  FF2 R;
  prod2(r, sp, R.h, R.l);
  float2 P, T;
  prod3(R, ct, P, T);
  const float2 x = add2(P, T);
  prod3(R, st, P, T);
  const float2 y = add2(P, T);
  prod2(r, cp, P, T);
  const float2 z = add2(P, T);
  X = fma2(x, make_float2(ft.cneg0 ? -1.0f : 1.0f, ft.cneg1 ? -1.0f : 1.0f), bc(0.0f));
  Y = fma2(y, make_float2(copysignf(1.0f, mt.x), copysignf(1.0f, mt.y)), bc(0.0f));
  Z = fma2(z, make_float2(pneg0 ? -1.0f : 1.0f, pneg1 ? -1.0f : 1.0f), bc(0.0f));
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
