// prngd_mrg.cuh -- one step of L'Ecuyer's MRG32k3a in exact 32/64-bit integer arithmetic
// (__host__ __device__, so the host tests can run it too).
#pragma once
#include <stdint.h>

#include "prngd_math.cuh"

namespace prngd {

constexpr uint32_t kMrgM1 = 4294967087u;  // 2^32 - 209
constexpr uint32_t kMrgM2 = 4294944443u;  // 2^32 - 22853

struct Mrg32k3a {
  uint32_t a0, a1, a2;  // x1_{n-3}, x1_{n-2}, x1_{n-1}
  uint32_t b0, b1, b2;  // x2_{n-3}, x2_{n-2}, x2_{n-1}
};

// v mod m1 for v < 2^54, folding 2^32 = 209 (mod m1) in 32-bit arithmetic: the high word times
// 209 is below 2^30, and a carry out of adding it to the low word (the sum then < 2^30) folds
// once more as + 209.
PRNGD_HD uint32_t mod_m1(uint64_t v) {
  const uint32_t t = (uint32_t)(v >> 32) * 209u;
  uint32_t r = (uint32_t)v + t;
  if (r < t) r += 209u;
  return r >= kMrgM1 ? r - kMrgM1 : r;
}
// v mod m2 for v < 2^54, folding 2^32 = 22853 (mod m2): after one wide fold w < 2^37, whose
// high word (< 32) folds with a 32-bit multiply; a carry out of that add (the sum then < 2^20)
// folds once more.
PRNGD_HD uint32_t mod_m2(uint64_t v) {
  const uint64_t w = (uint64_t)(uint32_t)(v >> 32) * 22853u + (uint32_t)v;  // one 32 x 32 -> 64 multiply-add
  const uint32_t t = (uint32_t)(w >> 32) * 22853u;  // < 2^20
  uint32_t r = (uint32_t)w + t;
  if (r < t) r += 22853u;
  return r >= kMrgM2 ? r - kMrgM2 : r;
}

// One step; returns z in [1, m1]. The negative terms are made positive by adding a multiple of
// the modulus: 1403580 x1_{n-2} + 810728 (m1 - x1_{n-3}) < 2^54, and likewise for x2.
PRNGD_HD uint32_t mrg_next(Mrg32k3a& g) {
  const uint32_t p1 = mod_m1((uint64_t)1403580u * g.a1 + (uint64_t)810728u * (kMrgM1 - g.a0));
  const uint32_t p2 = mod_m2((uint64_t)527612u * g.b2 + (uint64_t)1370589u * (kMrgM2 - g.b0));
  g.a0 = g.a1;
  g.a1 = g.a2;
  g.a2 = p1;
  g.b0 = g.b1;
  g.b1 = g.b2;
  g.b2 = p2;
  return p1 > p2 ? p1 - p2 : p1 - p2 + kMrgM1;
}

// Fast path of floor(V 2^64), V = n / D, D = (m1 - 1)^2 = (2^32 - 210)^2, n = A m1 + B < 2^64.
// With c = 210 2^-32, 2^64 / D = sum (i + 1) c^i, so with n = nh 2^32 + nl
//   V 2^64 = n + E0 + E1 2^-32 + E2 2^-64 + eps,
//   E0 = 420 nh, E1 = 420 nl + 132300 nh, E2 = 132300 nl + 37044000 nh,
// 0 <= eps < 5.4e-10 (37044000 nl 2^-96 and the terms from 5 c^4 n on). With S = E1 + (E2 >> 32)
// the exact value is n + E0 + (S + r) 2^-32 with 0 <= r < 3.3, so the integer part is
// n + E0 + (S >> 32) unless the low word of S lies within 16 of 2^32 (`ok` = 0). For A >= 2^22
// it is at least 2^54, and it rounds like the xorshift fast path's I.
PRNGD_HD uint64_t mrg_fast_I(uint64_t n, uint32_t& ok) {
  // the halves as 32-bit values, so that every product is one 32 x 32 -> 64 multiply(-add)
  const uint32_t nh = (uint32_t)(n >> 32), nl = (uint32_t)n;
  const uint64_t E0 = (uint64_t)nh * 420u;
  const uint64_t E1 = (uint64_t)nl * 420u + (uint64_t)nh * 132300u;
  const uint64_t E2 = (uint64_t)nl * 132300u + (uint64_t)nh * 37044000u;
  const uint64_t S = E1 + (E2 >> 32);
  ok = ((uint32_t)S < 0xFFFFFFF0u) ? 1u : 0u;
  return n + E0 + (S >> 32);
}

}  // namespace prngd
