// prngd_math.cuh -- per-output arithmetic of the PRNGD construction (arXiv:1401.8230,
// Section 2) for sm_103a: stream seeding, the xorshift128 base draws, the accept-reject
// test, and the three conversions of the exact value z' = n / D to output bits.
//
// Notation: u1, u2 are w-bit draws, A = u1 - 1, B = u2 + 1, n = A 2^w + B (Eq. 4 reduced),
// D = (2^w - 1)^2, V = n / D in [1/D, (D-1)/D]. V is never dyadic (D is odd and > n), so it
// is never a tie for any rounding and never exactly representable.
//
// All functions are __host__ __device__ so the arithmetic can be exercised off the GPU too.
#pragma once
#include <stdint.h>

#if defined(__CUDACC__)
#define PRNGD_HD __host__ __device__ __forceinline__
#else
#define PRNGD_HD inline
#endif

namespace prngd {

// ------------------------------------------------------------------------ bit helpers
PRNGD_HD int clz32(uint32_t v) {
#if defined(__CUDA_ARCH__)
  return __clz((int)v);
#else
  return v ? __builtin_clz(v) : 32;
#endif
}
PRNGD_HD int clz64(uint64_t v) {
#if defined(__CUDA_ARCH__)
  return __clzll((long long)v);
#else
  return v ? __builtin_clzll(v) : 64;
#endif
}
PRNGD_HD float bits_to_float(uint32_t v) {
#if defined(__CUDA_ARCH__)
  return __uint_as_float(v);
#else
  float f;
  __builtin_memcpy(&f, &v, 4);
  return f;
#endif
}
PRNGD_HD uint32_t float_to_bits(float f) {
#if defined(__CUDA_ARCH__)
  return __float_as_uint(f);
#else
  uint32_t v;
  __builtin_memcpy(&v, &f, 4);
  return v;
#endif
}
PRNGD_HD float int_to_float_rn(int32_t v) {
#if defined(__CUDA_ARCH__)
  return __int2float_rn(v);
#else
  return (float)v;
#endif
}
PRNGD_HD float fmul_rn(float a, float b) {
#if defined(__CUDA_ARCH__)
  return __fmul_rn(a, b);
#else
  return a * b;
#endif
}
// a * b + c with a 64-bit result (one wide multiply-add).
PRNGD_HD uint64_t mad_wide(uint32_t a, uint32_t b, uint64_t c) {
#if defined(__CUDA_ARCH__)
  uint64_t d;
  asm("mad.wide.u32 %0, %1, %2, %3;" : "=l"(d) : "r"(a), "r"(b), "l"(c));
  return d;
#else
  return (uint64_t)a * b + c;
#endif
}
// (hi:lo) >> s, low word, for 0 <= s < 32.
PRNGD_HD uint32_t funnel_r(uint32_t lo, uint32_t hi, uint32_t s) {
#if defined(__CUDA_ARCH__)
  return __funnelshift_r(lo, hi, s);
#else
  return (uint32_t)((((uint64_t)hi << 32) | lo) >> (s & 31));
#endif
}
PRNGD_HD uint64_t umulhi64(uint64_t a, uint64_t b) {
#if defined(__CUDA_ARCH__)
  return __umul64hi(a, b);
#else
  return (uint64_t)(((unsigned __int128)a * b) >> 64);
#endif
}

// ------------------------------------------------------------------------ base streams
// splitmix64 (Steele, Lea, Flood 2014): the k-th output (k = 0, 1, ...) of the sequence
// started at state `seed` is mix(seed + (k+1) * gamma), mix a bijective finaliser.
constexpr uint64_t kGoldenGamma = 0x9E3779B97F4A7C15ull;

PRNGD_HD uint64_t splitmix_finalise(uint64_t z) {
  z ^= z >> 30;
  z *= 0xBF58476D1CE4E5B9ull;
  z ^= z >> 27;
  z *= 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

struct XorShift128 {
  uint32_t x, y, z, w;
};

// Stream s of `seed` takes splitmix64 outputs 2s and 2s+1, low word first. The finaliser maps
// only 0 to 0 and its two inputs differ by gamma, so the state is never all zero.
PRNGD_HD XorShift128 seed_stream(uint64_t seed, uint64_t s) {
  const uint64_t o0 = splitmix_finalise(seed + (2 * s + 1) * kGoldenGamma);
  const uint64_t o1 = splitmix_finalise(seed + (2 * s + 2) * kGoldenGamma);
  return XorShift128{(uint32_t)o0, (uint32_t)(o0 >> 32), (uint32_t)o1, (uint32_t)(o1 >> 32)};
}

// Marsaglia (2003) xor128, shift triple (11, 8, 19); returns the new w word.
PRNGD_HD uint32_t xs_next(XorShift128& s) {
  const uint32_t t = s.x ^ (s.x << 11);
  s.x = s.y;
  s.y = s.z;
  s.z = s.w;
  s.w = s.w ^ (s.w >> 19) ^ (t ^ (t >> 8));
  return s.w;
}

// The inverse step: the state before the last xs_next. With (x, y, z, w) the current state,
// the previous one is (x0, x, y, z) where t = x0 ^ (x0 << 11) satisfies t ^ (t >> 8) =
// w ^ z ^ (z >> 19); both xor-shifts are inverted by repeating them until the shift passes
// 32 bits.
PRNGD_HD void xs_prev(XorShift128& s) {
  const uint32_t r = s.w ^ s.z ^ (s.z >> 19);
  const uint32_t t = r ^ (r >> 8) ^ (r >> 16) ^ (r >> 24);
  const uint32_t x0 = t ^ (t << 11) ^ (t << 22);
  s.w = s.z;
  s.z = s.y;
  s.y = s.x;
  s.x = x0;
}

// T^J s for g = x^J mod P, g given as four 32-bit words (bit i of the polynomial = bit i%32 of
// word i/32): the sum of T^i s over the set bits of g.
PRNGD_HD XorShift128 apply_poly(const uint32_t g[4], XorShift128 s) {
  XorShift128 acc{0u, 0u, 0u, 0u};
  for (int word = 0; word < 4; ++word) {
    uint32_t bits = g[word];
    for (int b = 0; b < 32; ++b) {
      const uint32_t m = 0u - (bits & 1u);  // all ones when the coefficient is set
      acc.x ^= s.x & m;
      acc.y ^= s.y & m;
      acc.z ^= s.z & m;
      acc.w ^= s.w & m;
      bits >>= 1;
      xs_next(s);
    }
  }
  return acc;
}

// A w-bit base draw: the top w bits of the 32-bit output (x = u 2^-w).
template <int W>
PRNGD_HD uint32_t draw(XorShift128& s, int w_rt) {
  const uint32_t r = xs_next(s);
  if constexpr (W == 32) {
    return r;
  } else if constexpr (W > 0) {
    return r >> (32 - W);
  } else {
    return w_rt == 32 ? r : r >> (32 - w_rt);
  }
}

// Accept-reject (Section 2): the pair is dropped when x1 = a0 (u1 = 0) or x1 = a
// (u1 = 2^w - 1). One unsigned compare: u1 - 1 < 2^w - 2.
PRNGD_HD bool accepted(uint32_t u1, uint32_t top /* 2^w - 1 */) { return (uint32_t)(u1 - 1u) < top - 1u; }

PRNGD_HD uint64_t numerator(uint32_t u1, uint32_t u2, int w) {
  return ((uint64_t)(u1 - 1u) << w) + (uint64_t)u2 + 1u;
}

// Double bits of n (n >= 1) rounded to nearest even, by integer operations: the FP64 unit's
// unsigned-to-double conversion runs at about half the rate of its multiply on this GPU.
// L = bit length of n; up to 53 bits the value is exact, above that n is cut at bit s = L - 53
// and rounded up when the cut part is more than half, or exactly half with an odd result.
// A mantissa that rounds up to 2^53 carries into the exponent.
PRNGD_HD uint64_t u64_to_f64_bits(uint64_t n) {
  const int L = 64 - clz64(n);
  if (L <= 53) return ((uint64_t)(L + 1021) << 52) + (n << (53 - L));
  const int s = L - 53;
  const uint64_t q = n >> s, rem = n & ((1ull << s) - 1), half = 1ull << (s - 1);
  const uint64_t up = (rem > half || (rem == half && (q & 1))) ? 1u : 0u;
  return ((uint64_t)(L + 1021) << 52) + q + up;
}

// ------------------------------------------------------------------------ exact division
// Constants for dividing by D without a hardware divide: D' = D << sh is D normalised to a
// set top bit, and v = floor((2^128 - 1) / D') - 2^64 is its Moller-Granlund reciprocal
// ("Improved division by invariant integers", IEEE Trans. Comput. 60(2), 2011, Alg. 4).
struct DivConst {
  uint64_t d_norm;  // D << sh
  uint64_t v;       // reciprocal
  int sh;           // 64 - 2w
};

// The constants for w = 32 and w = 24, fixed at compile time (D' = D 2^(64-2w); v as above; the
// host test recomputes both from the definition).
template <int W>
PRNGD_HD DivConst divconst_for() {
  static_assert(W == 32 || W == 24, "compile-time constants exist for w = 32 and w = 24");
  if constexpr (W == 32) {
    return DivConst{0xFFFFFFFE00000001ull, 0x200000003ull, 0};
  } else {
    return DivConst{0xFFFFFE0000010000ull, 0x20000030000ull, 16};
  }
}

// Double bits of RN(V) for any w in [2, 32], exactly. Normalise n to m = n 2^c in
// [2^63, 2^64); Y = m / D' lies in (1/2, 2) and V = Y 2^(sh - c). The 2-by-1 division of
// m 2^53 (Y >= 1) or m 2^54 (Y < 1) by D' gives the 54-bit integer part q of Y 2^53 or
// Y 2^54; V is never a tie, so rounding to nearest is "round up iff the last bit of q is set".
PRNGD_HD uint64_t rn_bits_exact(uint64_t n, const DivConst& dc) {
  const int c = clz64(n);
  const uint64_t m = n << c;
  const bool ge = m >= dc.d_norm;
  const int k = ge ? 53 : 54;
  const uint64_t u1 = m >> (64 - k);  // < 2^54 <= D'
  const uint64_t u0 = m << k;
  // Algorithm 4 (div 2-by-1): q = floor((u1 2^64 + u0) / D'), with the remainder's two
  // corrections.
  uint64_t q0 = dc.v * u1;
  uint64_t q1 = umulhi64(dc.v, u1);
  const uint64_t s0 = q0 + u0;
  q1 += u1 + (s0 < q0 ? 1u : 0u);
  q0 = s0;
  q1 += 1;
  uint64_t r = u0 - q1 * dc.d_norm;
  if (r > q0) {
    q1 -= 1;
    r += dc.d_norm;
  }
  if (r >= dc.d_norm) {
    q1 += 1;
    r -= dc.d_norm;
  }
  const uint64_t mant = (q1 >> 1) + (q1 & 1);  // in [2^52, 2^53]; 2^53 carries into the exponent
  const int e = dc.sh - c - (ge ? 0 : 1);       // unbiased exponent of V
  return ((uint64_t)(e + 1022) << 52) + mant;
}

// Double bits of RN(V) from I = floor(V 2^64) when I >= 2^54: the 54-bit integer part of
// V 2^(53 - L) is I >> (L - 53) (nested floors), L = bit length of I minus one.
PRNGD_HD uint64_t rn_bits_from_scaled(uint64_t I) {
  const uint32_t ihi = (uint32_t)(I >> 32);  // >= 2^22
  const int p = 31 - clz32(ihi);             // L - 32, in [22, 31]
  const uint64_t q = I >> (p - 21);          // in [2^53, 2^54)
  const uint64_t mant = (q >> 1) + (q & 1);
  return ((uint64_t)(p + 990) << 52) + mant;  // exponent L - 64, biased: L + 959, minus 1 for mant
}

// Fast path for w = 32. With eps = 2^-32,
//   V 2^64 = n / (1 - eps)^2 = A 2^32 + (B + 2A) + sum_{j>=1} ((j+1) B + (j+2) A) eps^j,
// and the tail beyond j = 1 is below 7.01 eps. With X = 2B + 3A (35 bits) the integer part is
// I = A 2^32 + B + 2A + (X >> 32) unless the low word of X is within 8 of 2^32. Needs
// A >= 2^22 so that I >= 2^54, and A <= 2^32 - 4 so that I + 2^10 < 2^64 (the largest values,
// which round to 1.0, take the exact path). fast32_ok says whether the fast path applies (it
// also rejects u1 = 0 and u1 = 2^32 - 1, which the caller's slow path handles).
PRNGD_HD uint64_t fast32_X(uint32_t u1, uint32_t u2) { return (uint64_t)u1 * 3u + (uint64_t)u2 * 2u - 1u; }
PRNGD_HD bool fast32_ok(uint32_t u1, uint64_t X) {
  return ((uint32_t)(u1 - 0x400001u) < 0xFFBFFFFDu) & ((uint32_t)X < 0xFFFFFFF8u);  // 2^22 <= A <= 2^32-4
}
PRNGD_HD uint64_t fast32_bits(uint32_t u1, uint32_t u2, uint64_t X) {
  // I = (u1 - 1) 2^32 + (2 u1 + u2 - 1 + (X >> 32)), in 32-bit words.
  const uint64_t L = (uint64_t)u1 * 2u + (uint64_t)u2 + (X >> 32) - 1u;  // < 2^35
  const uint32_t ilo = (uint32_t)L;
  const uint32_t ihi = (u1 - 1u) + (uint32_t)(L >> 32);  // >= 2^22
  // Round at bit s = L - 53 of I (L = 32 + p its top bit) by adding 2^s, then keep the 53 bits
  // above it; a carry out of the top is the next binade (exponent + 1, mantissa 0).
  const uint32_t p = 31u - (uint32_t)clz32(ihi);  // in [22, 31]
  const uint32_t s = p - 21u;                       // in [1, 10]
  const uint32_t jlo = ilo + (1u << s);
  const uint32_t jhi = ihi + (jlo < ilo ? 1u : 0u);
  const uint32_t mlo = funnel_r(jlo, jhi, s + 1u);
  const uint32_t mhi = (jhi >> (s + 1u)) + ((p + 990u) << 20);  // biased exponent L - 64, minus the implicit 1
  return ((uint64_t)mhi << 32) | mlo;
}

// Medium path for w = 32, small values: 1 <= A < 2^22, so I < 2^54 and the double needs bits
// below I. One more series term gives floor(V 2^96) = I 2^32 + (X mod 2^32) + (Y >> 32) with
// Y = 3B + 4A = X + u1 + u2 (35 bits), unless the low word of Y is within 16 of 2^32 (the
// remaining tail is below 10 2^-32). The 96-bit value is shifted left so its top bit is bit 95;
// the 54-bit integer part of V at its binade is then bits 95..42, rounded at bit 42 (V is
// never a tie). Valid when medium32_ok holds (the X condition of the fast path included).
PRNGD_HD bool medium32_ok(uint32_t u1, uint64_t X, uint32_t u2) {
  const uint64_t Y = X + (uint64_t)u1 + (uint64_t)u2;
  return ((uint32_t)(u1 - 2u) < 0x3FFFFFu) &  // 1 <= A < 2^22
         ((uint32_t)X < 0xFFFFFFF8u) & ((uint32_t)Y < 0xFFFFFFF0u);
}
// Double bits of RN(V) from T = floor(V 2^96) = t2 2^64 + t1 2^32 + t0 with 1 <= t2 < 2^23:
// shift T left so its top bit is bit 95; the 54-bit integer part of V at its binade is bits
// 95..42, rounded at bit 42 (V is never a tie).
PRNGD_HD uint64_t rn_bits_from_scaled96(uint32_t t2, uint32_t t1, uint32_t t0) {
  const uint32_t p = 31u - (uint32_t)clz32(t2);
  const uint32_t k = 31u - p;  // in [9, 31]
  const uint32_t n2 = (t2 << k) | (t1 >> (32u - k));
  const uint32_t n1 = (t1 << k) | (t0 >> (32u - k));
  const uint64_t q = ((((uint64_t)n2) << 32) | n1) >> 10;  // bits 95..42: in [2^53, 2^54)
  const uint64_t mant = (q >> 1) + (q & 1);               // in [2^52, 2^53]; 2^53 carries into the exponent
  return ((uint64_t)(p + 990u) << 52) + mant;             // V in [2^(p-32), 2^(p-31))
}

PRNGD_HD uint64_t medium32_bits(uint32_t u1, uint32_t u2, uint64_t X) {
  const uint64_t Y = X + (uint64_t)u1 + (uint64_t)u2;
  const uint64_t I = ((uint64_t)(u1 - 1u) << 32) + (uint64_t)u1 * 2u + (uint64_t)u2 - 1u + (X >> 32);
  // T = I 2^32 + xlo + (Y >> 32), as words t2 t1 t0
  const uint64_t low = (uint64_t)(uint32_t)X + (Y >> 32);
  const uint64_t mid = (I & 0xFFFFFFFFull) + (low >> 32);
  return rn_bits_from_scaled96((uint32_t)(I >> 32) + (uint32_t)(mid >> 32), (uint32_t)mid, (uint32_t)low);
}

// Fast path for w = 24. With eps = 2^-24,
//   V 2^64 = A 2^40 + (B + 2A) 2^16 + (2B + 3A) 2^-8 + (3B + 4A) 2^-32 + tail,
// tail < 9.01 2^-32. With K = (2B + 3A) 2^24 + (3B + 4A) (< 2^51) the integer part is
// I = A 2^40 + (B + 2A) 2^16 + (K >> 32) unless the low word of K is within 16 of 2^32.
// Needs A >= 2^14 so that I >= 2^54.
PRNGD_HD uint64_t fast24_K(uint32_t u1, uint32_t u2) {
  const uint32_t A = u1 - 1u, B = u2 + 1u;
  return ((uint64_t)(2u * B + 3u * A) << 24) + (uint64_t)(3u * B + 4u * A);
}
PRNGD_HD bool fast24_ok(uint32_t u1, uint64_t K) {
  return ((uint32_t)(u1 - 1u - 0x4000u) < 0xFFBFFEu) & ((uint32_t)K < 0xFFFFFFF0u);  // 2^14 <= A <= 2^24-3
}
PRNGD_HD uint64_t fast24_bits(uint32_t u1, uint32_t u2, uint64_t K) {
  const uint32_t A = u1 - 1u, B = u2 + 1u;
  // I = A 2^40 + (B + 2A) 2^16 + (K >> 32), in 32-bit words: the high word is A 2^8 plus the
  // carry out of the low 48-bit sum.
  const uint64_t L = ((uint64_t)(B + 2u * A) << 16) + (K >> 32);  // < 2^42
  const uint32_t ilo = (uint32_t)L;
  const uint32_t ihi = (A << 8) + (uint32_t)(L >> 32);  // >= 2^22
  const uint32_t p = 31u - (uint32_t)clz32(ihi);
  const uint32_t s = p - 21u;
  const uint32_t jlo = ilo + (1u << s);
  const uint32_t jhi = ihi + (jlo < ilo ? 1u : 0u);
  const uint32_t mlo = funnel_r(jlo, jhi, s + 1u);
  const uint32_t mhi = (jhi >> (s + 1u)) + ((p + 990u) << 20);
  return ((uint64_t)mhi << 32) | mlo;
}

// Medium path for w = 24, small values 1 <= A < 2^14 (I < 2^54): with c3 = 4B + 5A,
//   floor(V 2^96) = I 2^32 + (K mod 2^32) + floor(c3 / 2^24)
// unless the low 24 bits of c3 are within 16 of 2^24 (the tail is below 11.01 2^-24).
PRNGD_HD bool medium24_ok(uint32_t u1, uint64_t K, uint32_t u2) {
  const uint32_t c3 = 4u * u2 + 5u * u1 - 1u;  // 4B + 5A, < 2^28
  return ((uint32_t)(u1 - 2u) < 0x3FFFu) &     // 1 <= A < 2^14
         ((uint32_t)K < 0xFFFFFFF0u) & ((c3 & 0xFFFFFFu) < 0xFFFFF0u);
}
PRNGD_HD uint64_t medium24_bits(uint32_t u1, uint32_t u2, uint64_t K) {
  const uint32_t A = u1 - 1u, B = u2 + 1u;
  const uint32_t c3 = 4u * B + 5u * A;
  const uint64_t I = ((uint64_t)A << 40) + ((uint64_t)(B + 2u * A) << 16) + (K >> 32);
  const uint64_t low = (uint64_t)(uint32_t)K + (c3 >> 24);
  const uint64_t mid = (I & 0xFFFFFFFFull) + (low >> 32);
  return rn_bits_from_scaled96((uint32_t)(I >> 32) + (uint32_t)(mid >> 32), (uint32_t)mid, (uint32_t)low);
}

// ------------------------------------------------------------------------ Eq. 5 map
// Eq. 5 (one generator on [0, 1 - k]: Eq. 6) maps an accepted pair to
//   z' = (1 - k^2) m / (D - 2),   m = n - 1 = (u1 - 1) 2^w + u2 in [0, D - 2],
// and its complement 1 - z' = ((D - 2) 2^2w - (2^2w - 1) m) / ((D - 2) 2^2w). Both are never
// dyadic except at m = 0 and m = D - 2 (gcd(2^2w - 1, D - 2) = 1), so rounding to nearest is
// again "round up iff the round bit is set". E = D - 2 is odd.

// Division constants of E' = (D - 2) << sh (same construction as divconst_for).
template <int W>
PRNGD_HD DivConst divconst_eq5_for() {
  static_assert(W == 32 || W == 24, "compile-time constants exist for w = 32 and w = 24");
  if constexpr (W == 32) {
    return DivConst{0xFFFFFFFDFFFFFFFFull, 0x200000005ull, 0};
  } else {
    return DivConst{0xFFFFFDFFFFFF0000ull, 0x20000050000ull, 16};
  }
}

// q = floor((u1 2^64 + u0) / d), r = the remainder, for u1 < d and d normalised (Moller-Granlund
// 2-by-1 division with reciprocal v).
PRNGD_HD uint64_t div_2by1(uint64_t u1, uint64_t u0, uint64_t d, uint64_t v, uint64_t& r) {
  uint64_t q0 = v * u1;
  uint64_t q1 = umulhi64(v, u1);
  const uint64_t s0 = q0 + u0;
  q1 += u1 + (s0 < q0 ? 1u : 0u);
  q0 = s0;
  q1 += 1;
  uint64_t rr = u0 - q1 * d;
  if (rr > q0) {
    q1 -= 1;
    rr += d;
  }
  if (rr >= d) {
    q1 += 1;
    rr -= d;
  }
  r = rr;
  return q1;
}

// Double bits of RN(N / E) 2^-scale for a 128-bit N = nhi 2^64 + nlo with 1 <= N / E < 2^64
// and N / E never a tie (ec: the constants of E' = E << ec.sh). N 2^sh / E' has the same value;
// the first 2-by-1 division gives its integer part q1 (>= 1), a second one the next 64 bits.
// The 54-bit integer part of the quotient at its binade is taken from q1:q2 and rounded up iff
// its last bit is set. Returns 0 for N = 0.
PRNGD_HD uint64_t rn_bits_ratio128(uint64_t nhi, uint64_t nlo, const DivConst& ec, int scale) {
  if ((nhi | nlo) == 0) return 0;
  const uint64_t hi = ec.sh ? (nhi << ec.sh) | (nlo >> (64 - ec.sh)) : nhi;
  const uint64_t lo = nlo << ec.sh;
  uint64_t r1, r2;
  const uint64_t q1 = div_2by1(hi, lo, ec.d_norm, ec.v, r1);  // >= 1
  const uint64_t q2 = div_2by1(r1, 0, ec.d_norm, ec.v, r2);
  const int L1 = 64 - clz64(q1);  // bit length of q1, in [1, 64]
  uint64_t q;                     // 54-bit integer part of the quotient at its binade
  if (L1 >= 54) {
    q = q1 >> (L1 - 54);
  } else {
    const int t = 54 - L1;  // in [1, 53]
    q = (q1 << t) | (q2 >> (64 - t));
  }
  const uint64_t mant = (q >> 1) + (q & 1);  // in [2^52, 2^53]
  const int e = L1 - 1 - scale;              // unbiased exponent of the value
  return ((uint64_t)(e + 1022) << 52) + mant;
}

// Exact Eq. 5 value bits from the accepted pair (u1, u2) of w-bit draws (w in [2, 32]); ec: the
// constants of D - 2; one_minus selects 1 - z'.
PRNGD_HD uint64_t eq5_bits_exact_w(uint32_t u1, uint32_t u2, int w, const DivConst& ec, bool one_minus) {
  const uint64_t m = ((uint64_t)(u1 - 1u) << w) + u2;
  const int s2 = 2 * w;  // in [4, 64]
  // N = (2^2w - 1) m = m 2^2w - m, as 128-bit words
  uint64_t nhi = (s2 == 64) ? m : (m >> (64 - s2));
  uint64_t nlo = (s2 == 64) ? 0 : (m << s2);
  nhi -= (nlo < m) ? 1u : 0u;
  nlo -= m;
  if (one_minus) {
    if (m == 0) return 0x3FF0000000000000ull;  // 1 - 0 = 1 exactly (the quotient would be 2^2w)
    const uint64_t top = (w == 32) ? 0xFFFFFFFFull : ((1ull << w) - 1u);
    const uint64_t e = top * top - 2u;  // D - 2
    const uint64_t ehi = (s2 == 64) ? e : (e >> (64 - s2)), elo = (s2 == 64) ? 0 : (e << s2);
    const uint64_t lo = elo - nlo;
    nhi = ehi - nhi - (elo < nlo ? 1u : 0u);
    nlo = lo;
  }
  return rn_bits_ratio128(nhi, nlo, ec, s2);
}
template <int W>
PRNGD_HD uint64_t eq5_bits_exact(uint32_t u1, uint32_t u2, bool one_minus) {
  return eq5_bits_exact_w(u1, u2, W, divconst_eq5_for<W>(), one_minus);
}

// Fast path for Eq. 5 at w = 32. With delta = 2^-31 + 2^-64, D - 2 = 2^64 (1 - delta) and
//   (1 - 2^-64) / (1 - delta) = 1 + 2^-31 + 2^-62 + 1.25 2^-93 + O(2^-124)
// (the 2^-64 terms cancel), so z' 2^64 = m + 2A + u2 2^-31 + A 2^-30 + tail, A = u1 - 1, with a
// positive tail below 14 2^-32. With Y = 4A + 2 u2 (35 bits) the integer part is
//   I5 = A 2^32 + 2A + u2 + (Y >> 32)
// unless the low word of Y is within 64 of 2^32. The complement 1 - z' of the pair is
// z'(~u1, ~u2) + 2^-64: its integer part is I5 of the complemented draws plus 1. Needs
// 2^22 <= A <= 2^32 - 4 (as the Eq. 4 fast path).
PRNGD_HD uint64_t fast32_eq5_Y(uint32_t u1, uint32_t u2) {
  return ((uint64_t)(u1 - 1u) << 2) + ((uint64_t)u2 << 1);
}
PRNGD_HD bool fast32_eq5_ok(uint32_t u1, uint64_t Y) {
  return ((uint32_t)(u1 - 0x400001u) < 0xFFBFFFFDu) & ((uint32_t)Y < 0xFFFFFFC0u);
}
PRNGD_HD uint64_t fast32_eq5_bits(uint32_t u1, uint32_t u2, uint64_t Y, uint32_t plus) {
  const uint32_t A = u1 - 1u;
  const uint64_t L = (uint64_t)A * 2u + (uint64_t)u2 + (Y >> 32) + plus;  // < 2^35
  const uint32_t ilo = (uint32_t)L;
  const uint32_t ihi = A + (uint32_t)(L >> 32);  // >= 2^22
  const uint32_t p = 31u - (uint32_t)clz32(ihi);
  const uint32_t s = p - 21u;
  const uint32_t jlo = ilo + (1u << s);
  const uint32_t jhi = ihi + (jlo < ilo ? 1u : 0u);
  const uint32_t mlo = funnel_r(jlo, jhi, s + 1u);
  const uint32_t mhi = (jhi >> (s + 1u)) + ((p + 990u) << 20);
  return ((uint64_t)mhi << 32) | mlo;
}

// Medium path for Eq. 5 at w = 32, small values 1 <= A < 2^22 (I5 < 2^54). One more series
// term: z' 2^96 = I5 2^32 + (Y mod 2^32) + Z 2^-32 + tail with Z = 4 u2 + 10 A (35 bits) and
// a positive tail below 1.25 u2 2^-61 + 2^-38 < 10.01 2^-32, so
//   floor(z' 2^96) = I5 2^32 + (Y mod 2^32) + (Z >> 32)
// unless the low word of Z is within 16 of 2^32. The complement adds 2^-64, i.e. 1 to I5 of
// the complemented draws (plus = 1).
PRNGD_HD bool medium32_eq5_ok(uint32_t u1, uint32_t u2) {
  const uint64_t Z = ((uint64_t)u2 << 2) + 10u * (uint64_t)(u1 - 1u);
  return ((uint32_t)(u1 - 2u) < 0x3FFFFFu) & ((uint32_t)Z < 0xFFFFFFF0u);  // 1 <= A < 2^22
}
// The words t2 t1 t0 of floor(z' 2^96) (of the complement's, with plus = 1).
PRNGD_HD void medium32_eq5_words(uint32_t u1, uint32_t u2, uint64_t Y, uint32_t plus, uint32_t& t2, uint32_t& t1,
                                 uint32_t& t0) {
  const uint64_t A = u1 - 1u;
  const uint64_t Z = ((uint64_t)u2 << 2) + 10u * A;
  const uint64_t I = (A << 32) + 2u * A + u2 + (Y >> 32) + plus;
  const uint64_t low = (uint64_t)(uint32_t)Y + (Z >> 32);
  const uint64_t mid = (I & 0xFFFFFFFFull) + (low >> 32);
  t2 = (uint32_t)(I >> 32) + (uint32_t)(mid >> 32);
  t1 = (uint32_t)mid;
  t0 = (uint32_t)low;
}
PRNGD_HD uint64_t medium32_eq5_bits(uint32_t u1, uint32_t u2, uint64_t Y, uint32_t plus) {
  uint32_t t2, t1, t0;
  medium32_eq5_words(u1, u2, Y, plus, t2, t1, t0);
  return rn_bits_from_scaled96(t2, t1, t0);
}

// Fast path for Eq. 5 at w = 24. With delta = 2^-23 + 2^-48,
//   (1 - 2^-48) / (1 - delta) = 1 + 2^-23 + 2^-46 + 1.25 2^-69 + O(2^-92),
// so with m = A 2^24 + u2,
//   z' 2^64 = A 2^40 + (u2 + 2A) 2^16 + (2^25 u2 + 2^26 A + 4 u2 + 10 A) 2^-32 + tail,
// tail positive and below 27 2^-32. With K5 = 2^25 u2 + 2^26 A + 4 u2 + 10 A (< 2^51) the
// integer part is I5 = A 2^40 + (u2 + 2A) 2^16 + (K5 >> 32) unless the low word of K5 is
// within 64 of 2^32. The complement adds 2^-48, i.e. 2^16 to I5 of the complemented draws.
// Needs 2^14 <= A <= 2^24 - 3.
PRNGD_HD uint64_t fast24_eq5_K(uint32_t u1, uint32_t u2) {
  const uint64_t A = u1 - 1u;
  return ((uint64_t)u2 << 25) + (A << 26) + 4u * (uint64_t)u2 + 10u * A;
}
PRNGD_HD bool fast24_eq5_ok(uint32_t u1, uint64_t K) {
  return ((uint32_t)(u1 - 1u - 0x4000u) < 0xFFBFFEu) & ((uint32_t)K < 0xFFFFFFC0u);
}
// Medium path for Eq. 5 at w = 24 (1 <= A < 2^14, so m < 2^38). Exactly,
//   (1 - 2^-48) / (1 - 2^-23 - 2^-48) = 1 + 2^-23 + 2^-46 + 2^-69 + 2^-71 + 2^-92 + 2^-93 + r,
// 0 < r < 1.82 2^-115, so
//   z' 2^96 = m 2^48 + m 2^25 + 4m + G / 2^45 + R,   G = m (2^24 + 2^22 + 3) < 2^63,
// with 0 < R < 2^-28 for m < 2^38. floor(z' 2^96) is therefore the sum with floor(G / 2^45)
// unless the low 45 bits of G lie within 2^20 of 2^45. The complement adds 2^-48, i.e. 2^48.
PRNGD_HD bool medium24_eq5_ok(uint32_t u1, uint32_t u2) {
  const uint64_t m = ((uint64_t)(u1 - 1u) << 24) + u2;
  const uint64_t G = m * 0x1400003ull;
  return ((uint32_t)(u1 - 2u) < 0x3FFFu) & ((G & 0x1FFFFFFFFFFFull) < 0x1FFFFFF00000ull);  // 1 <= A < 2^14
}
// The words t2 t1 t0 of floor(z' 2^96) (of the complement's, with plus = 1).
PRNGD_HD void medium24_eq5_words(uint32_t u1, uint32_t u2, uint32_t plus, uint32_t& t2, uint32_t& t1,
                                 uint32_t& t0) {
  const uint64_t m = ((uint64_t)(u1 - 1u) << 24) + u2;
  const uint64_t G = m * 0x1400003ull;
  const uint64_t low = (m << 25) + 4u * m + (G >> 45) + ((uint64_t)plus << 48);  // < 2^64
  const uint64_t lo64 = ((m & 0xFFFFull) << 48) + low;
  t2 = (uint32_t)(m >> 16) + (lo64 < low ? 1u : 0u);
  t1 = (uint32_t)(lo64 >> 32);
  t0 = (uint32_t)lo64;
}
PRNGD_HD uint64_t medium24_eq5_bits(uint32_t u1, uint32_t u2, uint32_t plus) {
  uint32_t t2, t1, t0;
  medium24_eq5_words(u1, u2, plus, t2, t1, t0);
  return rn_bits_from_scaled96(t2, t1, t0);
}

// I = floor(z' 2^64) of the w = 24 Eq. 5 fast path (>= 2^54 when fast24_eq5_ok holds).
PRNGD_HD uint64_t fast24_eq5_I(uint32_t u1, uint32_t u2, uint64_t K, uint32_t plus) {
  const uint32_t A = u1 - 1u;
  const uint64_t L = ((uint64_t)(u2 + 2u * A) << 16) + (K >> 32) + plus;  // < 2^42
  return ((uint64_t)((A << 8) + (uint32_t)(L >> 32)) << 32) | (uint32_t)L;
}
PRNGD_HD uint64_t fast24_eq5_bits(uint32_t u1, uint32_t u2, uint64_t K, uint32_t plus) {
  const uint64_t I = fast24_eq5_I(u1, u2, K, plus);
  const uint32_t ilo = (uint32_t)I;
  const uint32_t ihi = (uint32_t)(I >> 32);  // >= 2^22
  const uint32_t p = 31u - (uint32_t)clz32(ihi);
  const uint32_t s = p - 21u;
  const uint32_t jlo = ilo + (1u << s);
  const uint32_t jhi = ihi + (jlo < ilo ? 1u : 0u);
  const uint32_t mlo = funnel_r(jlo, jhi, s + 1u);
  const uint32_t mhi = (jhi >> (s + 1u)) + ((p + 990u) << 20);
  return ((uint64_t)mhi << 32) | mlo;
}

// Form C from the form-B bits d: hi = RN32(d) by rounding the 53-bit significand to 24 bits
// (round half to even; d is dyadic so ties occur), lo = RN32(d - hi) where d - hi = R 2^(e-52)
// exactly for the signed integer R = (low 29 bits) - 2^29 * (rounded up). Packed as
// (lo bits << 32) | hi bits, i.e. hi first in memory.
PRNGD_HD uint64_t f32pair_from_bits(uint64_t d) {
  const uint32_t rem = (uint32_t)d & 0x1FFFFFFFu;
  const uint32_t top = (uint32_t)(d >> 29);  // sign | exp11 | 23 fraction bits
  const uint32_t up = (rem > 0x10000000u) || (rem == 0x10000000u && (top & 1u));
  const uint32_t hi = top - (896u << 23) + up;  // rebias 1023 -> 127
  const int32_t R = (int32_t)rem - (int32_t)(up << 29);
  const int e = (int)((d >> 52) & 0x7FF) - 1023;
  // lo = RN24(R) * 2^(e-52): the integer-to-float conversion rounds R to nearest even, and
  // the power-of-two scale is exact (e - 52 >= -116, inside the float normal range).
  const float scale = bits_to_float((uint32_t)(e - 52 + 127) << 23);
  const float lo = fmul_rn(int_to_float_rn(R), scale);
  return ((uint64_t)float_to_bits(lo) << 32) | hi;
}

}  // namespace prngd
