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

// The canonical residue of r < 2^32 modulo m = 2^32 - d (d < m): r - m wraps to r + d, which is
// larger than r exactly when r < m, so the smaller of the two is r mod m.
PRNGD_HD uint32_t canon(uint32_t r, uint32_t d) {
  const uint32_t s = r + d;
  return s < r ? s : r;
}
// v mod m1 for v < 2^54, folding 2^32 = 209 (mod m1) in 32-bit arithmetic: the high word times
// 209 is below 2^30, and a carry out of adding it to the low word (the sum then < 2^30) folds
// once more as + 209.
PRNGD_HD uint32_t mod_m1(uint64_t v) {
  const uint32_t t = (uint32_t)(v >> 32) * 209u;
  uint32_t r = (uint32_t)v + t;
  if (r < t) r += 209u;
  return canon(r, 209u);
}
// v mod m2 for v < 2^54, folding 2^32 = 22853 (mod m2): after one wide fold w < 2^37, whose
// high word (< 32) folds with a 32-bit multiply; a carry out of that add (the sum then < 2^20)
// folds once more.
PRNGD_HD uint32_t mod_m2(uint64_t v) {
  const uint64_t w = (uint64_t)(uint32_t)(v >> 32) * 22853u + (uint32_t)v;  // one 32 x 32 -> 64 multiply-add
  const uint32_t t = (uint32_t)(w >> 32) * 22853u;  // < 2^20
  uint32_t r = (uint32_t)w + t;
  if (r < t) r += 22853u;
  return canon(r, 22853u);
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

// Fast path of floor(V 2^64), V = n / D, D = (M - 1)^2, from A = u1 - 1 and B = u2 + 1
// (n = A M + B, M = m1) without forming n. With M - 1 = 2^32 (1 - c), c = 210 2^-32, V = A / (M - 1) + (A + B) / (M - 1)^2 expands as
//   V 2^64 = A 2^32 + (211 A + B) + (44520 A + 420 B) 2^-32 + (9393300 A + 132300 B) 2^-64 + R,
// every term of R positive and R 2^32 < 0.47 (largest at A = M - 3, B = M). With
// S = 44520 A + 420 B + ((9393300 A + 132300 B) >> 32) the part below 2^-32 adds less than 1.47
// to S, so floor(V 2^64) = A 2^32 + 211 A + B + (S >> 32) unless S's low word is within 16 of
// 2^32 (`ok` = 0). Every product is one 32 x 32 -> 64 multiply(-add). For A >= 2^22 the result
// is at least 2^54, and it rounds like the xorshift fast path's I.
PRNGD_HD uint64_t mrg_fast_I_ab(uint32_t A, uint32_t B, uint32_t& ok) {
  const uint64_t W = (uint64_t)A * 9393300u + (uint64_t)B * 132300u;
  const uint64_t S = (uint64_t)A * 44520u + (uint64_t)B * 420u + (uint32_t)(W >> 32);
  ok = ((uint32_t)S < 0xFFFFFFF0u) ? 1u : 0u;
  const uint64_t Y = (uint64_t)A * 211u + B + (uint32_t)(S >> 32);
  return ((uint64_t)A << 32) + Y;
}

}  // namespace prngd
