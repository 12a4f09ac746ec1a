// Host harness for the exact-decision arithmetic of the CUDA codec
// (paper_2003_02633_gb300/csrc/ivc_exact.cuh, compiled here as plain C++).
// Reads one command per line on stdin, writes one result line per command:
//   P den                  -> m e              (pi / den)
//   S m D                  -> cm ce cx sm se sx cneg sneg   (cos, sin of pi m / D)
//   N xbits ybits zbits rbits -> bits          (RN32 norm from candidate r32)
//   R m e exact            -> bits             (round away from zero)
//   F hbits lbits          -> m e exact neg    (|h + l|)
//   M m1 e1 x1 m2 e2 x2    -> m e exact        (product)
//   A m1 e1 x1 m2 e2 x2    -> m e exact        (sum)
#define __host__
#define __device__
#define __forceinline__ inline
#include <cinttypes>
#include <cstdio>
#include <cstring>

#include "../paper_2003_02633_gb300/csrc/ivc_exact.cuh"

using namespace ivc::exact;

static float fbits(uint32_t b) {
  float f;
  memcpy(&f, &b, 4);
  return f;
}
static uint32_t bitsf(float f) {
  uint32_t b;
  memcpy(&b, &f, 4);
  return b;
}

int main() {
  char op[8];
  while (scanf("%7s", op) == 1) {
    if (op[0] == 'P') {
      long long den;
      if (scanf("%lld", &den) != 1) return 1;
      uint64_t m;
      int32_t e;
      pi_over_host(den, m, e);
      printf("%" PRIu64 " %d\n", m, e);
    } else if (op[0] == 'S') {
      int m, D;
      if (scanf("%d %d", &m, &D) != 2) return 1;
      uint64_t km;
      int32_t ke;
      pi_over_host(2LL * D, km, ke);
      SF c, s;
      bool cn, sn;
      sincospi_grid(m, D, SF{km, ke, false}, c, s, cn, sn);
      printf("%" PRIu64 " %d %d %" PRIu64 " %d %d %d %d\n", c.m, c.e, (int)c.exact, s.m, s.e,
             (int)s.exact, (int)cn, (int)sn);
    } else if (op[0] == 'N') {
      uint32_t xb, yb, zb, rb;
      if (scanf("%u %u %u %u", &xb, &yb, &zb, &rb) != 4) return 1;
      printf("%u\n", bitsf(norm_rn(fbits(xb), fbits(yb), fbits(zb), fbits(rb))));
    } else if (op[0] == 'R') {
      uint64_t m;
      int e, x;
      if (scanf("%" SCNu64 " %d %d", &m, &e, &x) != 3) return 1;
      printf("%u\n", bitsf(ra32(SF{m, e, x != 0})));
    } else if (op[0] == 'F') {
      uint32_t hb, lb;
      if (scanf("%u %u", &hb, &lb) != 2) return 1;
      bool neg;
      const SF v = sf_from_ff(fbits(hb), fbits(lb), neg);
      printf("%" PRIu64 " %d %d %d\n", v.m, v.e, (int)v.exact, (int)neg);
    } else if (op[0] == 'M' || op[0] == 'A') {
      uint64_t m1, m2;
      int e1, x1, e2, x2;
      if (scanf("%" SCNu64 " %d %d %" SCNu64 " %d %d", &m1, &e1, &x1, &m2, &e2, &x2) != 6)
        return 1;
      const SF a{m1, e1, x1 != 0}, b{m2, e2, x2 != 0};
      const SF r = op[0] == 'M' ? sf_mul(a, b) : sf_add(a, b);
      printf("%" PRIu64 " %d %d\n", r.m, r.e, (int)r.exact);
    } else {
      return 2;
    }
  }
  return 0;
}
