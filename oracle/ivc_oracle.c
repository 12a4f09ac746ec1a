/*
 * Oracle for inline 3-vector compression (Trojak & Witherden, "Inline Vector
 * Compression for Computational Physics", arXiv:2003.02633).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is a plain, slow, CPU implementation of
 * what the compressed-vector hot path computes.  Only the test suite, the
 * smoke check and the CPU-baseline leg of the benchmark may load it.  It shares
 * no code, header, table or constant generator with the CUDA library.
 *
 * Arithmetic: FP64, with a binary128 (_Float128) re-evaluation of every
 * decision that FP64 cannot settle (a bin decision within 1e-7 bin of a
 * rounding boundary, or a decoded value within 2^-44 relative of an FP32
 * rounding boundary).  The magnitude is always computed in binary128.
 *
 * Section references are to the paper.
 *   Sec. 2.1, Eq. (cart2sphere)/(spherical): r = |x|, theta = atan(y/x) in
 *            [-pi, pi), phi = acos(z/r) in [0, pi].
 *   Sec. 2.1, Eq. (a_disc): n = nint(n_max * psi), nint = round half up.
 *   Sec. 2.1, Eq. (a_inv): theta^ = pi(2 n_theta / n_theta_max - 1),
 *            phi^ = pi n_phi / n_phi_max.
 *   Sec. 2.3: sign bit of r dropped; E8 -> E7 with bias b7 (E^8 = E7 + b8 - b7);
 *            mantissa tail bit d23 dropped (truncation, rebuilt as zero);
 *            values below the range clamp to the lowest supported value.
 *   Fig. (comp_regimes): bit layouts <s,e,m>-p-t, fields from MSB: sign,
 *            exponent, mantissa, n_phi, n_theta.
 *   Sec. 2.4, Eq. (q_split): fractional splitting n_p = n_phi (n_theta_max+1)
 *            + n_theta.
 *   Sec. 2.5: tanh companding n = nint(m n_max [tanh(gamma(2 psi - 1)) + c]),
 *            c = tanh(gamma), m = 1/(2c).
 *   Sec. 2.4, Eq. (stat): e_i = |x_i - x^_i|_2, mean, sample deviation.
 *   Sec. 5: C = A + B on decompressed vectors, result recompressed.
 *
 * Readings where the paper is silent (each also listed in the design notes):
 *   - r is rounded to FP32 from the exact norm (RN32(|x|)); its mantissa is
 *     then truncated to the layout's width.
 *   - phi is evaluated as atan2(sqrt(x^2+y^2), z), identical to acos(z/r) in
 *     exact arithmetic and well conditioned near the poles.
 *   - exponent field 0 is the zero vector; the all-ones field is reserved for
 *     non-finite words; normal fields are 1 .. 2^e - 2.
 *   - below range: clamp to (E=1, m=0) (default) or flush to the zero word;
 *     above range: saturate to (E=2^e-2, m=all ones) (default) or the
 *     all-ones exponent with m=0 (infinite magnitude).
 *   - NaN anywhere: all-ones exponent, m=1, angles 0.  Infinite components:
 *     direction taken from the infinite components, magnitude overflows.
 *   - n_theta = n_theta_max (theta = pi, the same direction as -pi) is stored
 *     as 0; at the poles (n_phi = 0 or n_phi_max) n_theta is stored as 0.
 *   - decoding computes r^ cos/sin products exactly and rounds each component
 *     away from zero to FP32 (exact zeros decode as +0).
 *   - the fused operations round in FP32: add is a + b, axpy is fmaf(alpha,
 *     x, y), the pointwise update is fmaf(dt, f, v) and m = rho * v.
 */
#define __STDC_WANT_IEC_60559_TYPES_EXT__
#define _GNU_SOURCE
#include <math.h>
#include <stdint.h>
#include <string.h>

typedef _Float128 quad;

static const quad QPI = 3.14159265358979323846264338327950288419716939937510582097494459F128;

/* ---------------------------------------------------------------- format */

typedef struct {
  int32_t sign_bits;      /* 0 or 1: a stored (always zero) sign bit of r    */
  int32_t exp_bits;       /* e: exponent width                               */
  int32_t man_bits;       /* m: mantissa width (<= 23)                       */
  int32_t phi_bits;       /* p                                               */
  int32_t theta_bits;     /* t                                               */
  int32_t exp_bias;       /* b_e (80 for the 7-bit exponent, 127 for 8-bit)  */
  int32_t map;            /* 0 uniform, 1 tanh companding, 2 fractional split */
  int32_t underflow_mode; /* 0 clamp to lowest value, 1 flush to zero        */
  int32_t overflow_mode;  /* 0 saturate, 1 infinite-magnitude code           */
  int32_t pad_;
  double gamma;           /* tanh companding strength                        */
  int64_t nphi_max_p1;    /* fractional split: n_phi_max + 1                 */
} ivco_format;

typedef struct {
  int64_t n_overflow, n_underflow, n_nonfinite, n_quad_angle, n_quad_decode;
} ivco_counts;

/* Derived quantities of a format. */
typedef struct {
  int64_t N;      /* n_theta_max */
  int64_t M;      /* n_phi_max   */
  int shift_m, shift_e, shift_s, shift_phi;
  uint64_t mask_theta, mask_phi, mask_m, mask_e, mask_np;
  int64_t e_max_field;  /* 2^e - 1 */
} layout;

static int make_layout(const ivco_format *f, layout *L) {
  int total = f->sign_bits + f->exp_bits + f->man_bits + f->phi_bits + f->theta_bits;
  if (total > 64 || f->exp_bits < 2 || f->exp_bits > 8 || f->man_bits < 1 ||
      f->man_bits > 23 || f->phi_bits < 1 || f->theta_bits < 1 ||
      f->sign_bits < 0 || f->sign_bits > 1)
    return -1;
  L->shift_phi = f->theta_bits;
  L->shift_m = f->theta_bits + f->phi_bits;
  L->shift_e = L->shift_m + f->man_bits;
  L->shift_s = L->shift_e + f->exp_bits;
  L->mask_theta = (1ull << f->theta_bits) - 1;
  L->mask_phi = (1ull << f->phi_bits) - 1;
  L->mask_m = (1ull << f->man_bits) - 1;
  L->mask_e = (1ull << f->exp_bits) - 1;
  L->mask_np = (f->phi_bits + f->theta_bits >= 64) ? ~0ull
               : ((1ull << (f->phi_bits + f->theta_bits)) - 1);
  L->e_max_field = (int64_t)L->mask_e;
  if (f->map == 2) {
    /* Eq. (q_split): (n_phi_max+1)(n_theta_max+1) - 1 < 2^p, p = phi+theta bits */
    int P = f->phi_bits + f->theta_bits;
    if (P > 62 || f->nphi_max_p1 < 2) return -1;
    int64_t cap = (int64_t)1 << P;
    L->M = f->nphi_max_p1 - 1;
    L->N = cap / f->nphi_max_p1 - 1;
    if (L->N < 1) return -1;
  } else {
    L->N = ((int64_t)1 << f->theta_bits) - 1;
    L->M = ((int64_t)1 << f->phi_bits) - 1;
  }
  return 0;
}

/* ---------------------------------------------------------- quantisation */

/* psi -> pre-rounding bin coordinate t (Eq. a_disc, or the tanh map of
 * Sec. 2.5).  psi = 1/2 exactly maps to n_max/2 exactly for both maps. */
static double t_of_psi_d(const ivco_format *f, double psi, int64_t nmax) {
  if (f->map == 1) {
    if (psi == 0.5) return 0.5 * (double)nmax;
    double c = tanh(f->gamma);
    return (double)nmax * (tanh(f->gamma * (2.0 * psi - 1.0)) + c) / (2.0 * c);
  }
  return (double)nmax * psi;
}

static quad t_of_psi_q(const ivco_format *f, quad psi, int64_t nmax) {
  if (f->map == 1) {
    if (psi == 0.5F128) return 0.5F128 * (quad)nmax;
    quad g = (quad)f->gamma;
    quad c = tanhf128(g);
    return (quad)nmax * (tanhf128(g * (2 * psi - 1)) + c) / (2 * c);
  }
  return (quad)nmax * psi;
}

/* nint(t) = floor(t + 1/2): round half up (Sec. 2.1). */
static int64_t nint_d(double t) { return (int64_t)floor(t + 0.5); }
static int64_t nint_q(quad t) { return (int64_t)floorf128(t + 0.5F128); }

static int near_half(double t) {
  double fr = t - floor(t);
  return fabs(fr - 0.5) < 1e-7;
}

/* Bin indices of a direction (X, Y, Z), not all zero.
 *
 * t is evaluated in FP64.  Within 1e-7 bin of a boundary k + 1/2 the decision
 * is re-taken: exactly (a sign test) when the boundary angle is a multiple of
 * pi/2, where FP32 inputs can sit arbitrarily close to it, else in binary128. */
static void quantise_angles(const ivco_format *f, const layout *L, double X,
                            double Y, double Z, int64_t *n_theta,
                            int64_t *n_phi, ivco_counts *cnt) {
  /* theta = atan2(y, x) in [-pi, pi]; exactly 0 on the positive x half-axis */
  double th = (Y == 0.0 && X > 0.0) ? 0.0 : atan2(Y, X);
  double psi_t = (Y == 0.0 && X > 0.0) ? 0.5 : 0.5 + th / (2.0 * M_PI);
  double tt = t_of_psi_d(f, psi_t, L->N);
  int64_t nt;
  if (near_half(tt)) {
    int64_t k = (int64_t)floor(tt);       /* boundary at t = k + 1/2 */
    int64_t h2 = 2 * k + 1;               /* 2 t_h */
    int uni = (f->map != 1);
    if (cnt) cnt->n_quad_angle++;
    if (h2 == L->N)                                   /* theta_h = 0     */
      nt = (Y >= 0.0) ? k + 1 : k;
    else if (uni && 2 * h2 == L->N)                   /* theta_h = -pi/2 */
      nt = (X >= 0.0) ? k + 1 : k;
    else if (uni && 2 * h2 == 3 * L->N)               /* theta_h = +pi/2 */
      nt = (X <= 0.0) ? k + 1 : k;
    else {
      quad thq = atan2f128((quad)Y, (quad)X);
      nt = nint_q(t_of_psi_q(f, 0.5F128 + thq / (2 * QPI), L->N));
    }
  } else {
    nt = nint_d(tt);
  }
  /* phi = acos(z/r) = atan2(rho, z); exactly pi/2 when z = 0 */
  double rho = sqrt(X * X + Y * Y);
  double ph = (Z == 0.0) ? 0.5 * M_PI : atan2(rho, Z);
  double psi_p = (Z == 0.0) ? 0.5 : ph / M_PI;
  double tp = t_of_psi_d(f, psi_p, L->M);
  int64_t np;
  if (near_half(tp)) {
    int64_t k = (int64_t)floor(tp);
    if (cnt) cnt->n_quad_angle++;
    if (2 * k + 1 == L->M)                            /* phi_h = pi/2    */
      np = (Z <= 0.0) ? k + 1 : k;
    else {
      quad rq = sqrtf128((quad)X * (quad)X + (quad)Y * (quad)Y);
      np = nint_q(t_of_psi_q(f, atan2f128(rq, (quad)Z) / QPI, L->M));
    }
  } else {
    np = nint_d(tp);
  }
  if (nt < 0) nt = 0;
  if (nt > L->N) nt = L->N;
  if (np < 0) np = 0;
  if (np > L->M) np = L->M;
  /* canonical forms: theta = pi is theta = -pi; theta is void at the poles */
  if (nt == L->N) nt = 0;
  if (np == 0 || np == L->M) nt = 0;
  *n_theta = nt;
  *n_phi = np;
}

static uint64_t pack(const ivco_format *f, const layout *L, int64_t E,
                     int64_t m, int64_t nt, int64_t np) {
  uint64_t w = ((uint64_t)E << L->shift_e) | ((uint64_t)m << L->shift_m);
  if (f->map == 2)
    w |= (uint64_t)(np * (L->N + 1) + nt);       /* Eq. (q_split) */
  else
    w |= ((uint64_t)np << L->shift_phi) | (uint64_t)nt;
  (void)f;
  return w;  /* sign bit of r, when present, is always 0 */
}

static uint32_t f32_bits(float v) { uint32_t u; memcpy(&u, &v, 4); return u; }

/* Compress one FP32 3-vector into a word (Sec. 2, Sec. 3). */
uint64_t ivco_encode(const ivco_format *f, float x, float y, float z,
                     ivco_counts *cnt) {
  layout L;
  if (make_layout(f, &L)) return 0;
  if (isnan(x) || isnan(y) || isnan(z)) {
    if (cnt) cnt->n_nonfinite++;
    return ((uint64_t)L.e_max_field << L.shift_e) | (1ull << L.shift_m);
  }
  if (x == 0.0f && y == 0.0f && z == 0.0f) return 0;
  int inf_in = isinf(x) || isinf(y) || isinf(z);
  double X = x, Y = y, Z = z;
  if (inf_in) {
    X = isinf(x) ? copysign(1.0, x) : copysign(0.0, x);
    Y = isinf(y) ? copysign(1.0, y) : copysign(0.0, y);
    Z = isinf(z) ? copysign(1.0, z) : copysign(0.0, z);
  }
  int64_t nt, np;
  quantise_angles(f, &L, X, Y, Z, &nt, &np, cnt);

  /* magnitude: r32 = RN32(|x|), exact norm evaluated in binary128 */
  int64_t E, m;
  int over = inf_in, under = 0;
  if (!inf_in) {
    quad s = (quad)x * (quad)x + (quad)y * (quad)y + (quad)z * (quad)z;
    float r32 = (float)sqrtf128(s);
    uint32_t u = f32_bits(r32);
    int64_t E8 = (u >> 23) & 0xff;
    int64_t M23 = u & 0x7fffff;
    if (E8 == 255) {
      over = 1;
      E = 0; m = 0;
    } else if (E8 == 0) {
      under = 1;
      E = 0; m = 0;
    } else {
      E = E8 - 127 + f->exp_bias;   /* E^8 = E_e + b8 - b_e */
      m = M23 >> (23 - f->man_bits); /* drop the tail bits (truncation) */
      if (E < 1) under = 1;
      if (E > L.e_max_field - 1) over = 1;
    }
  } else {
    E = 0; m = 0;
  }
  if (under) {
    if (cnt) cnt->n_underflow++;
    if (f->underflow_mode == 1) return 0;
    E = 1; m = 0;
  }
  if (over) {
    if (cnt) cnt->n_overflow++;
    if (f->overflow_mode == 1) { E = L.e_max_field; m = 0; }
    else { E = L.e_max_field - 1; m = (int64_t)L.mask_m; }
  }
  return pack(f, &L, E, m, nt, np);
}

/* ---------------------------------------------------------------- decode */

/* sin(pi a / b), cos(pi a / b) for integers a, b > 0: exact reduction to
 * |r| <= 1/4 by the nearest multiple of 1/2, then FP64 (or binary128). */
static void sincospi_rat_d(int64_t a, int64_t b, double *s, double *c) {
  int64_t twob = 2 * b;
  int64_t am = a % twob;
  if (am < 0) am += twob;                      /* a/b mod 2 in [0, 2) */
  int64_t j = (2 * am) / b;                    /* j = nearest integer to 2a/b */
  int64_t num = 2 * am - j * b;
  if (2 * num > b) { j++; num -= b; }          /* r = num / (2b), |r| <= 1/4 */
  double sr, cr;
  if (num == 0) { sr = 0.0; cr = 1.0; }
  else {
    double r = (double)num / (double)twob;
    sr = sin(M_PI * r);
    cr = cos(M_PI * r);
  }
  switch (j & 3) {
    case 0: *s = sr;  *c = cr;  break;
    case 1: *s = cr;  *c = -sr; break;
    case 2: *s = -sr; *c = -cr; break;
    default: *s = -cr; *c = sr; break;
  }
}

static void sincospi_rat_q(int64_t a, int64_t b, quad *s, quad *c) {
  int64_t twob = 2 * b;
  int64_t am = a % twob;
  if (am < 0) am += twob;
  int64_t j = (2 * am) / b;
  int64_t num = 2 * am - j * b;
  if (2 * num > b) { j++; num -= b; }
  quad sr, cr;
  if (num == 0) { sr = 0; cr = 1; }
  else {
    quad r = (quad)num / (quad)twob;
    sr = sinf128(QPI * r);
    cr = cosf128(QPI * r);
  }
  switch (j & 3) {
    case 0: *s = sr;  *c = cr;  break;
    case 1: *s = cr;  *c = -sr; break;
    case 2: *s = -sr; *c = -cr; break;
    default: *s = -cr; *c = sr; break;
  }
}

/* psi^ of the tanh map (inverse of Sec. 2.5), in binary128; the end points
 * and the centre are exact. */
static quad psi_hat_tanh_q(const ivco_format *f, int64_t n, int64_t nmax) {
  if (n == 0) return 0;
  if (n == nmax) return 1;
  if (2 * n == nmax) return 0.5F128;
  quad g = (quad)f->gamma;
  quad c = tanhf128(g);
  quad w = c * (2 * (quad)n / (quad)nmax - 1);
  return 0.5F128 * (1 + atanhf128(w) / g);
}

/* Angles of a word as (sin, cos) pairs, in FP64 (uniform map only) and in
 * binary128. */
static void angles_d(const layout *L, int64_t nt, int64_t np, double *st,
                     double *ct, double *sp, double *cp) {
  /* theta^ = pi (2 n_theta - N) / N ; phi^ = pi n_phi / M   (Eq. a_inv) */
  sincospi_rat_d(2 * nt - L->N, L->N, st, ct);
  sincospi_rat_d(np, L->M, sp, cp);
}

static void angles_q(const ivco_format *f, const layout *L, int64_t nt,
                     int64_t np, quad *st, quad *ct, quad *sp, quad *cp) {
  if (f->map == 1) {
    quad pt = psi_hat_tanh_q(f, nt, L->N);
    quad pp = psi_hat_tanh_q(f, np, L->M);
    /* theta^ = pi (2 psi^ - 1), phi^ = pi psi^ */
    if (pt == 0 || pt == 1 || pt == 0.5F128)
      sincospi_rat_q(pt == 0 ? -1 : (pt == 1 ? 1 : 0), 1, st, ct);
    else {
      quad th = QPI * (2 * pt - 1);
      *st = sinf128(th); *ct = cosf128(th);
    }
    if (pp == 0 || pp == 1 || pp == 0.5F128)
      sincospi_rat_q(pp == 0 ? 0 : (pp == 1 ? 2 : 1), 2, sp, cp);
    else {
      quad ph = QPI * pp;
      *sp = sinf128(ph); *cp = cosf128(ph);
    }
    return;
  }
  sincospi_rat_q(2 * nt - L->N, L->N, st, ct);
  sincospi_rat_q(np, L->M, sp, cp);
}

/* Round a real value away from zero to FP32 (exact zero -> +0). */
static float ra32_d(double v) {
  if (v == 0.0) return 0.0f;
  float f = (float)v;
  if ((double)f != v && fabs((double)f) < fabs(v))
    f = nextafterf(f, v > 0 ? INFINITY : -INFINITY);
  return f;
}

static float ra32_q(quad v) {
  if (v == 0) return 0.0f;
  float f = (float)v;
  quad fq = (quad)f;
  if (fq != v && fabsf128(fq) < fabsf128(v))
    f = nextafterf(f, v > 0 ? INFINITY : -INFINITY);
  return f;
}

/* Is an FP64 value too close to an FP32 rounding boundary (the FP32 grid
 * itself, for directed rounding) to trust its FP64 error? */
static int near_f32_grid(double v) {
  if (v == 0.0) return 0;
  float f = (float)v;
  if (isinf(f)) return 0;
  double d = fabs(v - (double)f);
  return d <= ldexp(fabs(v), -44);
}

static void unpack(const ivco_format *f, const layout *L, uint64_t w,
                   int64_t *E, int64_t *m, int64_t *nt, int64_t *np) {
  *E = (int64_t)((w >> L->shift_e) & L->mask_e);
  *m = (int64_t)((w >> L->shift_m) & L->mask_m);
  if (f->map == 2) {
    uint64_t npk = w & L->mask_np;
    *np = (int64_t)(npk / (uint64_t)(L->N + 1));
    *nt = (int64_t)(npk % (uint64_t)(L->N + 1));
  } else {
    *np = (int64_t)((w >> L->shift_phi) & L->mask_phi);
    *nt = (int64_t)(w & L->mask_theta);
  }
}

/* Decompress one word (Eq. a_inv and Eq. cart2sphere), rounding away from
 * zero to FP32. */
void ivco_decode(const ivco_format *f, uint64_t w, float out[3],
                 ivco_counts *cnt) {
  layout L;
  if (make_layout(f, &L)) { out[0] = out[1] = out[2] = NAN; return; }
  int64_t E, m, nt, np;
  unpack(f, &L, w, &E, &m, &nt, &np);
  if (E == 0) { out[0] = out[1] = out[2] = 0.0f; return; }
  if (E == L.e_max_field) {
    if (m != 0) { out[0] = out[1] = out[2] = NAN; return; }
    quad st, ct, sp, cp;
    angles_q(f, &L, nt, np, &st, &ct, &sp, &cp);
    quad d[3] = {ct * sp, st * sp, cp};
    for (int i = 0; i < 3; i++)
      out[i] = d[i] == 0 ? 0.0f : (d[i] > 0 ? INFINITY : -INFINITY);
    return;
  }
  /* r^ = 2^(E - b_e) (1 + m / 2^man): exact in FP64 and binary128 */
  double r = ldexp(1.0 + ldexp((double)m, -f->man_bits), (int)(E - f->exp_bias));
  if (f->map != 1) {
    double st, ct, sp, cp;
    angles_d(&L, nt, np, &st, &ct, &sp, &cp);
    double v[3] = {r * ct * sp, r * st * sp, r * cp};
    int risky = near_f32_grid(v[0]) || near_f32_grid(v[1]) || near_f32_grid(v[2]);
    if (!risky) {
      for (int i = 0; i < 3; i++) out[i] = ra32_d(v[i]);
      return;
    }
  }
  if (cnt) cnt->n_quad_decode++;
  quad st, ct, sp, cp;
  angles_q(f, &L, nt, np, &st, &ct, &sp, &cp);
  quad rq = (quad)r;
  quad v[3] = {rq * ct * sp, rq * st * sp, rq * cp};
  for (int i = 0; i < 3; i++) out[i] = ra32_q(v[i]);
}

/* Unrounded decode in FP64 (for error statistics). */
void ivco_decode_exact(const ivco_format *f, uint64_t w, double out[3]) {
  layout L;
  if (make_layout(f, &L)) { out[0] = out[1] = out[2] = NAN; return; }
  int64_t E, m, nt, np;
  unpack(f, &L, w, &E, &m, &nt, &np);
  if (E == 0) { out[0] = out[1] = out[2] = 0.0; return; }
  if (E == L.e_max_field) { out[0] = out[1] = out[2] = NAN; return; }
  double r = ldexp(1.0 + ldexp((double)m, -f->man_bits), (int)(E - f->exp_bias));
  quad st, ct, sp, cp;
  angles_q(f, &L, nt, np, &st, &ct, &sp, &cp);
  out[0] = (double)((quad)r * ct * sp);
  out[1] = (double)((quad)r * st * sp);
  out[2] = (double)((quad)r * cp);
}

/* Fields of a word: E, m, n_theta, n_phi (after the split, for map 2). */
void ivco_fields(const ivco_format *f, uint64_t w, int64_t out[4]) {
  layout L;
  if (make_layout(f, &L)) { out[0] = out[1] = out[2] = out[3] = -1; return; }
  unpack(f, &L, w, &out[0], &out[1], &out[2], &out[3]);
}

/* Derived n_theta_max, n_phi_max of a format (-1 if the format is invalid). */
void ivco_nmax(const ivco_format *f, int64_t out[2]) {
  layout L;
  if (make_layout(f, &L)) { out[0] = out[1] = -1; return; }
  out[0] = L.N;
  out[1] = L.M;
}

/* Pre-rounding bin coordinates t_theta, t_phi of a vector (binary128). */
void ivco_bin_coords(const ivco_format *f, float x, float y, float z,
                     double out[2]) {
  layout L;
  if (make_layout(f, &L)) { out[0] = out[1] = NAN; return; }
  quad X = x, Y = y, Z = z;
  quad pt = (y == 0.0f && x > 0.0f) ? 0.5F128
                                    : 0.5F128 + atan2f128(Y, X) / (2 * QPI);
  quad rho = sqrtf128(X * X + Y * Y);
  quad pp = (z == 0.0f) ? 0.5F128 : atan2f128(rho, Z) / QPI;
  out[0] = (double)t_of_psi_q(f, pt, L.N);
  out[1] = (double)t_of_psi_q(f, pp, L.M);
}

/* ------------------------------------------------------- array operations */

void ivco_compress(const ivco_format *f, const float *xyz, int64_t n,
                   uint64_t *w, ivco_counts *cnt) {
  for (int64_t i = 0; i < n; i++)
    w[i] = ivco_encode(f, xyz[3 * i], xyz[3 * i + 1], xyz[3 * i + 2], cnt);
}

void ivco_decompress(const ivco_format *f, const uint64_t *w, int64_t n,
                     float *xyz, ivco_counts *cnt) {
  for (int64_t i = 0; i < n; i++) ivco_decode(f, w[i], xyz + 3 * i, cnt);
}

/* Sec. 5: decompress two words, add in FP32, compress the sum. */
void ivco_add(const ivco_format *f, const uint64_t *a, const uint64_t *b,
              uint64_t *c, int64_t n, ivco_counts *cnt) {
  for (int64_t i = 0; i < n; i++) {
    float u[3], v[3];
    ivco_decode(f, a[i], u, cnt);
    ivco_decode(f, b[i], v, cnt);
    float s0 = u[0] + v[0], s1 = u[1] + v[1], s2 = u[2] + v[2];
    c[i] = ivco_encode(f, s0, s1, s2, cnt);
  }
}

/* y <- compress(fmaf(alpha, x^, y^)) */
void ivco_axpy(const ivco_format *f, float alpha, const uint64_t *x,
               uint64_t *y, int64_t n, ivco_counts *cnt) {
  for (int64_t i = 0; i < n; i++) {
    float u[3], v[3];
    ivco_decode(f, x[i], u, cnt);
    ivco_decode(f, y[i], v, cnt);
    float s0 = fmaf(alpha, u[0], v[0]);
    float s1 = fmaf(alpha, u[1], v[1]);
    float s2 = fmaf(alpha, u[2], v[2]);
    y[i] = ivco_encode(f, s0, s1, s2, cnt);
  }
}

/* v_out <- compress(fmaf(dt, f^, v^)); optionally m_out <- compress(rho v_new) */
void ivco_update(const ivco_format *f, float dt, const uint64_t *v,
                 const uint64_t *frc, const float *rho, uint64_t *v_out,
                 uint64_t *m_out, int64_t n, ivco_counts *cnt) {
  for (int64_t i = 0; i < n; i++) {
    float u[3], g[3];
    ivco_decode(f, v[i], u, cnt);
    ivco_decode(f, frc[i], g, cnt);
    float s0 = fmaf(dt, g[0], u[0]);
    float s1 = fmaf(dt, g[1], u[1]);
    float s2 = fmaf(dt, g[2], u[2]);
    v_out[i] = ivco_encode(f, s0, s1, s2, cnt);
    if (m_out && rho) {
      float q = rho[i];
      m_out[i] = ivco_encode(f, q * s0, q * s1, q * s2, cnt);
    }
  }
}

/* ---------------------------------------------------------- statistics */

typedef struct {
  double mean, sd, max;          /* Eq. (stat) on e_i = |x_i - x^_i|         */
  double mean_rel, max_rel;      /* e_i / |x_i| (Sec. 3 normalisation)       */
  double max_ang, rms_ang;       /* angle between x_i and x^_i (radians)     */
  double max_mag_rel, rms_mag_rel; /* | |x^_i| - |x_i| | / |x_i|             */
  int64_t n;
} ivco_stats;

/* Error of x^ (FP32, as stored) against x (FP32 inputs), all in FP64, for the
 * nonzero finite inputs.  x^ is given as an array (decode output or a plain
 * FP32/FP16/BF16 store converted back to FP32). */
void ivco_error_stats(const float *x, const float *xh, int64_t n,
                      ivco_stats *st) {
  double s = 0, s2 = 0, mx = 0, sr = 0, mr = 0, ma = 0, sa = 0, mm = 0, sm = 0;
  int64_t k = 0;
  for (int64_t i = 0; i < n; i++) {
    double a0 = x[3 * i], a1 = x[3 * i + 1], a2 = x[3 * i + 2];
    double b0 = xh[3 * i], b1 = xh[3 * i + 1], b2 = xh[3 * i + 2];
    if (!isfinite(a0) || !isfinite(a1) || !isfinite(a2)) continue;
    double na = sqrt(a0 * a0 + a1 * a1 + a2 * a2);
    if (na == 0.0) continue;
    double d0 = a0 - b0, d1 = a1 - b1, d2 = a2 - b2;
    double e = sqrt(d0 * d0 + d1 * d1 + d2 * d2);
    double nb = sqrt(b0 * b0 + b1 * b1 + b2 * b2);
    double cx0 = a1 * b2 - a2 * b1, cx1 = a2 * b0 - a0 * b2, cx2 = a0 * b1 - a1 * b0;
    double cr = sqrt(cx0 * cx0 + cx1 * cx1 + cx2 * cx2);
    double dt = a0 * b0 + a1 * b1 + a2 * b2;
    double ang = atan2(cr, dt);
    double mrel = fabs(nb - na) / na;
    s += e; s2 += e * e; if (e > mx) mx = e;
    sr += e / na; if (e / na > mr) mr = e / na;
    if (ang > ma) ma = ang;
    sa += ang * ang;
    if (mrel > mm) mm = mrel;
    sm += mrel * mrel;
    k++;
  }
  st->n = k;
  if (k == 0) { memset(st, 0, sizeof(*st)); return; }
  st->mean = s / k;
  st->sd = k > 1 ? sqrt(fmax(0.0, (s2 - s * s / k) / (k - 1))) : 0.0;
  st->max = mx;
  st->mean_rel = sr / k;
  st->max_rel = mr;
  st->max_ang = ma;
  st->rms_ang = sqrt(sa / k);
  st->max_mag_rel = mm;
  st->rms_mag_rel = sqrt(sm / k);
}
