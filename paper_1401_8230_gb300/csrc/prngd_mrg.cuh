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

// v mod m1 for v < 2^54, folding 2^32 = 209 (mod m1) twice.
PRNGD_HD uint32_t mod_m1(uint64_t v) {
  v = (v >> 32) * 209u + (v & 0xFFFFFFFFull);  // < 2^32 + 2^30
  v = (v >> 32) * 209u + (v & 0xFFFFFFFFull);  // < 2^32 + 209
  return (uint32_t)(v >= kMrgM1 ? v - kMrgM1 : v);
}
// v mod m2 for v < 2^54, folding 2^32 = 22853 (mod m2).
PRNGD_HD uint32_t mod_m2(uint64_t v) {
  v = (v >> 32) * 22853u + (v & 0xFFFFFFFFull);  // < 2^37
  v = (v >> 32) * 22853u + (v & 0xFFFFFFFFull);  // < 2^32 + 2^19
  return (uint32_t)(v >= kMrgM2 ? v - kMrgM2 : v);
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

}  // namespace prngd
