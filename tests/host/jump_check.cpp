// Host-compiled check of the library's xorshift128 jump (prngd_gf2.h, apply_poly of
// prngd_math.cuh): prints the characteristic polynomial it finds, then compares jumps of many
// sizes with plain stepping and checks that jumps compose. Built and run by test_host_jump.py.
#include <cstdint>
#include <cstdio>
#include <random>

#include "prngd_gf2.h"

using namespace prngd;
using namespace prngd_host;

int main() {
  Poly p;
  if (!find_charpoly(&p)) {
    printf("charpoly not found\n");
    return 1;
  }
  printf("charpoly %016llx %016llx\n", (unsigned long long)p.hi, (unsigned long long)p.lo);
  std::mt19937_64 rng(7);
  long bad = 0, checked = 0;
  // jumps against stepping, from random states
  for (uint64_t J : {0ull, 1ull, 2ull, 3ull, 127ull, 128ull, 129ull, 1000ull, 4096ull, 65535ull, 1000003ull, 33554432ull}) {
    for (int t = 0; t < 3; ++t) {
      XorShift128 a{(uint32_t)rng(), (uint32_t)rng(), (uint32_t)rng(), (uint32_t)rng()}, b = a;
      uint32_t g[4];
      words_of(x_pow_mod(J, p), g);
      const XorShift128 j = apply_poly(g, a);
      for (uint64_t k = 0; k < J; ++k) xs_next(b);
      ++checked;
      if (j.x != b.x || j.y != b.y || j.z != b.z || j.w != b.w) ++bad;
    }
  }
  // composition: x^a x^b = x^(a+b) and jump(a) after jump(b) = jump(a + b), at huge sizes
  for (int t = 0; t < 200; ++t) {
    const uint64_t A = rng() >> 2, B = rng() >> 2;
    const Poly ga = x_pow_mod(A, p), gb = x_pow_mod(B, p), gab = x_pow_mod(A + B, p);
    const Poly prod = mulmod_p(ga, gb, p);
    ++checked;
    if (prod.lo != gab.lo || prod.hi != gab.hi) ++bad;
    uint32_t wa[4], wb[4], wab[4];
    words_of(ga, wa);
    words_of(gb, wb);
    words_of(gab, wab);
    XorShift128 s{(uint32_t)rng(), (uint32_t)rng(), (uint32_t)rng(), 1u};
    const XorShift128 two = apply_poly(wa, apply_poly(wb, s)), one = apply_poly(wab, s);
    ++checked;
    if (two.x != one.x || two.y != one.y || two.z != one.z || two.w != one.w) ++bad;
  }
  // the period: x^(2^128 - 1) = 1, written as x^(2^64)^(2^64) x^-1; check x^(2^128) = x by
  // repeated squaring of x (128 squarings)
  {
    Poly q{2, 0};
    for (int i = 0; i < 128; ++i) q = mulmod_p(q, q, p);
    ++checked;
    if (q.lo != 2 || q.hi != 0) ++bad;
  }
  printf("checked %ld bad %ld\n", checked, bad);
  return bad != 0;
}
