// Pair decode of the fast path with the poles of the sphere settled in place.
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
  decode2<G>(w0, w1, tab_t, tab_p, F.Kt_h, F.Kt_l, F.Kp_h, F.Kp_l, X, Y, Z, s0, s1);
  if (s0) pole_or_generic<G>(w0, F, tab_t, tab_p, X.x, Y.x, Z.x);
  if (s1) pole_or_generic<G>(w1, F, tab_t, tab_p, X.y, Y.y, Z.y);
}

}  // namespace fast
}  // namespace ivc
