// prngd_gf2.h -- polynomials over GF(2) for the xorshift128 jump (host code).
//
// The step T of xorshift128 is linear over GF(2). Its characteristic polynomial P has degree
// 128; Berlekamp-Massey recovers it from 512 bits of one output bit of any nonzero state (the
// polynomial is primitive, so the bit sequence has no shorter recurrence). For a jump of J
// draws, g = x^J mod P gives T^J = g(T) (Cayley-Hamilton).
#pragma once
#include <stdint.h>

#include <vector>

#include "prngd_math.cuh"

namespace prngd_host {

struct Poly {  // coefficients of x^0 .. x^127 (P itself: x^128 + this)
  uint64_t lo, hi;
};

// a * b mod P, P = x^128 + p: Horner over the bits of b, multiplying by x and reducing.
inline Poly mulmod_p(const Poly& a, const Poly& b, const Poly& p) {
  Poly r{0, 0};
  for (int i = 127; i >= 0; --i) {
    const bool top = (r.hi >> 63) & 1;
    r.hi = (r.hi << 1) | (r.lo >> 63);
    r.lo <<= 1;
    if (top) {
      r.lo ^= p.lo;
      r.hi ^= p.hi;
    }
    const uint64_t bit = (i >= 64) ? (b.hi >> (i - 64)) & 1 : (b.lo >> i) & 1;
    if (bit) {
      r.lo ^= a.lo;
      r.hi ^= a.hi;
    }
  }
  return r;
}

// x^J mod P by squaring and multiplying.
inline Poly x_pow_mod(uint64_t J, const Poly& p) {
  Poly result{1, 0}, base{2, 0};  // 1 and x
  while (J) {
    if (J & 1) result = mulmod_p(result, base, p);
    base = mulmod_p(base, base, p);
    J >>= 1;
  }
  return result;
}

inline void words_of(const Poly& q, uint32_t g[4]) {
  g[0] = (uint32_t)q.lo;
  g[1] = (uint32_t)(q.lo >> 32);
  g[2] = (uint32_t)q.hi;
  g[3] = (uint32_t)(q.hi >> 32);
}

// Berlekamp-Massey over GF(2): the shortest recurrence s_n = sum_{i=1..L} c_i s_{n-i} of bit 0
// of 512 outputs; P(x) = x^L + sum c_i x^(L-i). Returns false unless L = 128 and the jumps it
// gives (1 and 1000 draws) equal plain stepping.
inline bool find_charpoly(Poly* out) {
  const int N = 512;
  std::vector<int> s(N);
  prngd::XorShift128 st{123456789u, 362436069u, 521288629u, 88675123u};
  for (int n = 0; n < N; ++n) s[n] = (int)(prngd::xs_next(st) & 1u);
  std::vector<int> C(N + 1, 0), B(N + 1, 0), T;
  C[0] = B[0] = 1;
  int L = 0, m = 1;
  for (int n = 0; n < N; ++n) {
    int d = s[n];
    for (int i = 1; i <= L; ++i) d ^= C[i] & s[n - i];
    if (!d) {
      ++m;
    } else if (2 * L <= n) {
      T = C;
      for (int i = 0; i + m <= N; ++i) C[i + m] ^= B[i];
      L = n + 1 - L;
      B = T;
      m = 1;
    } else {
      for (int i = 0; i + m <= N; ++i) C[i + m] ^= B[i];
      ++m;
    }
  }
  if (L != 128) return false;
  Poly p{0, 0};
  for (int d = 0; d < 128; ++d) {
    if (!C[128 - d]) continue;
    if (d < 64) p.lo |= 1ull << d;
    else p.hi |= 1ull << (d - 64);
  }
  for (uint64_t J : {1ull, 1000ull}) {
    uint32_t g[4];
    words_of(x_pow_mod(J, p), g);
    prngd::XorShift128 a{0x9E3779B9u, 0x7F4A7C15u, 0xF39CC060u, 0x5CEDC834u}, b = a;
    const prngd::XorShift128 j = prngd::apply_poly(g, a);
    for (uint64_t k = 0; k < J; ++k) prngd::xs_next(b);
    if (j.x != b.x || j.y != b.y || j.z != b.z || j.w != b.w) return false;
  }
  *out = p;
  return true;
}

}  // namespace prngd_host
