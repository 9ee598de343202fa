// Host-compiled check of the per-output arithmetic of the CUDA library (prngd_math.cuh is
// __host__ __device__) against the oracle, on cases random streams almost never reach: values
// near the fast paths' low-word boundaries, small values for the medium paths, and 96-bit
// values whose rounding carries into the next binade. Built and run by test_host_math.py.
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <random>

#include "prngd_math.cuh"

extern "C" {
double orc_value_rn(uint64_t n, int w);
uint64_t orc_numerator(uint32_t u1, uint32_t u2, int w);
int orc_accept(uint32_t u1, int w);
void orc_value_form_c(uint64_t n, int w, float* hi, float* lo);
int orc_values_mode(const uint32_t* u1, const uint32_t* u2, uint64_t count, int w, int form, int mode, void* out);
}

using namespace prngd;

static uint64_t bits_of(double d) {
  uint64_t b;
  memcpy(&b, &d, 8);
  return b;
}
static DivConst make_dc(int w) {
  const uint64_t m = (w == 32) ? 0xFFFFFFFFull : ((1ull << w) - 1);
  DivConst dc;
  dc.sh = 64 - 2 * w;
  dc.d_norm = (m * m) << dc.sh;
  const unsigned __int128 all = ~(unsigned __int128)0;
  dc.v = (uint64_t)(all / dc.d_norm - ((unsigned __int128)1 << 64));
  return dc;
}
static DivConst make_dc_eq5(int w) {
  const uint64_t m = (w == 32) ? 0xFFFFFFFFull : ((1ull << w) - 1);
  const uint64_t e = m * m - 2;
  DivConst dc;
  dc.sh = clz64(e);
  dc.d_norm = e << dc.sh;
  const unsigned __int128 all = ~(unsigned __int128)0;
  dc.v = (uint64_t)(all / dc.d_norm - ((unsigned __int128)1 << 64));
  return dc;
}
static long bad = 0, checked = 0;
static void expect(uint64_t got, uint64_t want, const char* what, uint32_t a, uint32_t b) {
  ++checked;
  if (got != want) {
    if (bad < 10) printf("%s u1=%u u2=%u got %016llx want %016llx\n", what, a, b, (unsigned long long)got,
                         (unsigned long long)want);
    ++bad;
  }
}
static uint64_t want_rn(uint32_t u1, uint32_t u2, int w) { return bits_of(orc_value_rn(orc_numerator(u1, u2, w), w)); }

// "words" mode: for each line "u1 u2 plus" on stdin print the 96-bit words of the Eq. 5
// medium path (t2 t1 t0), for an exact comparison with big-integer arithmetic.
// "words24": the same for the w = 24 medium path.
static int words_mode(bool w24) {
  unsigned long long a, b, c;
  while (scanf("%llu %llu %llu", &a, &b, &c) == 3) {
    uint32_t t2, t1, t0;
    if (w24)
      medium24_eq5_words((uint32_t)a, (uint32_t)b, (uint32_t)c, t2, t1, t0);
    else
      medium32_eq5_words((uint32_t)a, (uint32_t)b, fast32_eq5_Y((uint32_t)a, (uint32_t)b), (uint32_t)c, t2, t1, t0);
    printf("%u %u %u\n", t2, t1, t0);
  }
  return 0;
}

int main(int argc, char** argv) {
  if (argc > 1 && strcmp(argv[1], "words") == 0) return words_mode(false);
  if (argc > 1 && strcmp(argv[1], "words24") == 0) return words_mode(true);
  std::mt19937_64 rng(2024);
  // 0. the compile-time division constants equal the ones derived at run time
  {
    const DivConst a = make_dc(32), b = divconst_for<32>(), c = make_dc(24), d = divconst_for<24>();
    expect(a.d_norm == b.d_norm && a.v == b.v && a.sh == b.sh, 1, "divconst32", 32, 0);
    expect(c.d_norm == d.d_norm && c.v == d.v && c.sh == d.sh, 1, "divconst24", 24, 0);
  }
  // 1. exact division, every w, random and edge draws; form C from the exact bits
  for (int w = 2; w <= 32; ++w) {
    const DivConst dc = make_dc(w);
    const uint32_t top = (w == 32) ? 0xFFFFFFFFu : ((1u << w) - 1u);
    for (int i = 0; i < 20000; ++i) {
      uint32_t u1 = (uint32_t)rng() & top, u2 = (uint32_t)(rng() >> 32) & top;
      if (i < 16) {
        const uint32_t e[4] = {1u, 2u, top - 1u, top / 2u};
        u1 = e[i & 3];
        u2 = (i >> 2) == 0 ? 0u : ((i >> 2) == 1 ? top : (i >> 2) == 2 ? 1u : top - 1u);
      }
      if (!orc_accept(u1, w)) {
        if (accepted(u1, top)) expect(1, 0, "accept", u1, u2);
        continue;
      }
      const uint64_t n = numerator(u1, u2, w);
      expect(n, orc_numerator(u1, u2, w), "numerator", u1, u2);
      const uint64_t want = want_rn(u1, u2, w);
      expect(rn_bits_exact(n, dc), want, "exact", u1, u2);
      float h, l;
      orc_value_form_c(n, w, &h, &l);
      uint32_t hb, lb;
      memcpy(&hb, &h, 4);
      memcpy(&lb, &l, 4);
      expect(f32pair_from_bits(want), ((uint64_t)lb << 32) | hb, "form C", u1, u2);
    }
  }
  // 2. w = 32 fast path near the low-word boundary of X = 3 u1 + 2 u2 - 1, and the medium path
  //    for small u1 near the low-word boundary of Y = X + u1 + u2
  for (int it = 0; it < 200000; ++it) {
    const uint32_t u1 = (it & 1) ? 2u + (uint32_t)(rng() % ((1u << 22) - 2u)) : 0x400001u + (uint32_t)(rng() % 0xFFB00000u);
    for (int d = -12; d < 12; ++d) {
      const int64_t target = ((int64_t)(1 + rng() % 4) << 32) + d;
      const int64_t num = target + 1 - ((it & 1) ? 4 : 3) * (int64_t)u1;
      const int div = (it & 1) ? 3 : 2;
      if (num < 0 || num % div) continue;
      const int64_t u2l = num / div;
      if (u2l > 0xFFFFFFFFll) continue;
      const uint32_t u2 = (uint32_t)u2l;
      const uint64_t X = fast32_X(u1, u2);
      if (fast32_ok(u1, X)) expect(fast32_bits(u1, u2, X), want_rn(u1, u2, 32), "fast32", u1, u2);
      if (medium32_ok(u1, X, u2)) expect(medium32_bits(u1, u2, X), want_rn(u1, u2, 32), "medium32", u1, u2);
    }
  }
  // 3. w = 24: every u1 below 2^14 + 16 with random u2 (medium and fast), K and c3 boundaries
  for (uint32_t u1 = 0; u1 < (1u << 14) + 16; ++u1)
    for (int k = 0; k < 64; ++k) {
      const uint32_t u2 = (uint32_t)(rng() & 0xFFFFFF);
      const uint64_t K = fast24_K(u1, u2);
      if (fast24_ok(u1, K)) expect(fast24_bits(u1, u2, K), want_rn(u1, u2, 24), "fast24", u1, u2);
      if (medium24_ok(u1, K, u2)) expect(medium24_bits(u1, u2, K), want_rn(u1, u2, 24), "medium24", u1, u2);
    }
  for (int it = 0; it < 200000; ++it) {
    const uint32_t u1 = 2u + (uint32_t)(rng() % ((1u << 24) - 4u));
    const int64_t target = ((int64_t)(1 + rng() % 3) << 24) + (int64_t)(rng() % 40) - 20;
    const int64_t num = target + 1 - 5 * (int64_t)u1;
    if (num < 0 || num % 4 || num / 4 > 0xFFFFFF) continue;
    const uint32_t u2 = (uint32_t)(num / 4);
    const uint64_t K = fast24_K(u1, u2);
    if (fast24_ok(u1, K)) expect(fast24_bits(u1, u2, K), want_rn(u1, u2, 24), "fast24", u1, u2);
    if (medium24_ok(u1, K, u2)) expect(medium24_bits(u1, u2, K), want_rn(u1, u2, 24), "medium24", u1, u2);
  }
  // 4. the 96-bit rounding on constructed values, including all-ones mantissas whose rounding
  //    carries into the next binade; V lies strictly inside (T, T + 1) 2^-96 (never a tie)
  for (int p = 0; p <= 22; ++p)
    for (int v = 0; v < 4000; ++v) {
      uint32_t t2 = (1u << p) | ((uint32_t)rng() & ((1u << p) - 1u)), t1 = (uint32_t)rng(), t0 = (uint32_t)rng();
      if (v < 32) {
        t2 = (2u << p) - 1u;
        t1 = 0xFFFFFFFFu;
        t0 = 0xFFFFFFFFu - (uint32_t)v * 7u;
      }
      const unsigned __int128 T = ((unsigned __int128)t2 << 64) | ((unsigned __int128)t1 << 32) | t0;
      const int bl = 64 + p + 1;
      const int s = bl - 54;
      const unsigned __int128 q = T >> s;
      uint64_t m = (uint64_t)(q >> 1) + (uint64_t)(q & 1);  // round bit set: V above the midpoint
      const uint64_t want = ((uint64_t)(bl - 1 - 96 + 1022) << 52) + m;
      expect(rn_bits_from_scaled96(t2, t1, t0), want, "scaled96", t2, t1);
    }
  // 4b. unsigned 64-bit to double, round to nearest even, against the host's IEEE conversion:
  //     exact ties at every cut position, values around powers of two, random values
  {
    auto check = [&](uint64_t n) {
      const double d = (double)n;
      expect(u64_to_f64_bits(n), bits_of(d), "u64_to_f64", (uint32_t)(n >> 32), (uint32_t)n);
    };
    for (int s = 1; s <= 11; ++s)
      for (int k = 0; k < 2000; ++k) {
        const uint64_t q = (1ull << 52) | (rng() & ((1ull << 52) - 1));  // 53-bit head
        if ((q << s) >> s != q) continue;
        const uint64_t base = q << s, half = 1ull << (s - 1);
        const uint64_t ds[5] = {half - 1, half, half + 1, 0, (1ull << s) - 1};
        for (uint64_t d : ds) check(base + d);
      }
    for (int L = 1; L <= 64; ++L)
      for (int64_t d = -3; d <= 3; ++d) {
        const uint64_t p2 = (L == 64) ? 0 : (1ull << L);
        const uint64_t n = p2 + (uint64_t)d;
        if (n) check(n);
      }
    check(~0ull);
    for (int i = 0; i < 200000; ++i) check((rng() >> (rng() % 64)) | 1u);
  }
  // 5. Eq. 5 and 1 - z: constants, the exact 128-bit path and the fast paths against the oracle
  {
    const DivConst a = make_dc_eq5(32), b = divconst_eq5_for<32>(), c = make_dc_eq5(24), d = divconst_eq5_for<24>();
    expect(a.d_norm == b.d_norm && a.v == b.v && a.sh == b.sh, 1, "divconst_eq5_32", 32, 0);
    expect(c.d_norm == d.d_norm && c.v == d.v && c.sh == d.sh, 1, "divconst_eq5_24", 24, 0);
  }
  auto want_mode = [](uint32_t u1, uint32_t u2, int w, int mode) {
    double v;
    orc_values_mode(&u1, &u2, 1, w, 1, mode, &v);
    return bits_of(v);
  };
  for (int w : {32, 24}) {
    const uint32_t top = (w == 32) ? 0xFFFFFFFFu : 0xFFFFFFu;
    for (int i = 0; i < 300000; ++i) {
      uint32_t u1 = 1u + (uint32_t)(rng() % (top - 1u)), u2 = (uint32_t)rng() & top;
      if (i < 64) {  // end points, small and large values
        const uint32_t e1[8] = {1u, 1u, 2u, top - 1u, top - 1u, top - 2u, 3u, top / 2u};
        u1 = e1[i & 7];
        u2 = (i >> 3) & 1 ? top : (uint32_t)(i >> 4);
      } else if (i % 3 == 0) {
        u1 = 1u + (uint32_t)(rng() % ((w == 32) ? (1u << 23) : (1u << 15)));  // small A
      }
      for (int om = 0; om < 2; ++om) {
        const uint64_t want = want_mode(u1, u2, w, 1 | (om << 1));
        const uint64_t ex = (w == 32) ? eq5_bits_exact<32>(u1, u2, om) : eq5_bits_exact<24>(u1, u2, om);
        expect(ex, want, om ? "eq5 exact 1-z" : "eq5 exact", u1, u2);
        const uint32_t a1 = om ? (top - u1) : u1, a2 = om ? (top - u2) : u2;  // complemented draws
        if (w == 32) {
          const uint64_t Y = fast32_eq5_Y(a1, a2);
          if (fast32_eq5_ok(a1, Y)) expect(fast32_eq5_bits(a1, a2, Y, om), want, "fast32_eq5", u1, u2);
        } else {
          const uint64_t K = fast24_eq5_K(a1, a2);
          if (fast24_eq5_ok(a1, K)) expect(fast24_eq5_bits(a1, a2, K, om ? 0x10000u : 0u), want, "fast24_eq5", u1, u2);
        }
      }
      // Eq. 4 complement: the Eq. 4 arithmetic on the complemented draws
      const uint64_t want_c = want_mode(u1, u2, w, 2);
      expect(rn_bits_exact(numerator(top - u1, top - u2, w), make_dc(w)), want_c, "eq4 1-z", u1, u2);
    }
  }
  // fast32_eq5 near the low-word boundary of Y = 4A + 2 u2, both maps
  for (int it = 0; it < 200000; ++it) {
    const uint32_t u1 = 0x400001u + (uint32_t)(rng() % 0xFFB00000u);
    const int64_t A = (int64_t)u1 - 1;
    for (int dd = -80; dd < 8; dd += 2) {
      const int64_t target = ((int64_t)(1 + rng() % 4) << 32) + dd;
      const int64_t num = target - 4 * A;
      if (num < 0 || (num & 1) || num / 2 > 0xFFFFFFFFll) continue;
      const uint32_t u2 = (uint32_t)(num / 2);
      const uint64_t Y = fast32_eq5_Y(u1, u2);
      if (!fast32_eq5_ok(u1, Y)) continue;
      expect(fast32_eq5_bits(u1, u2, Y, 0), want_mode(u1, u2, 32, 1), "fast32_eq5 edge", u1, u2);
      expect(fast32_eq5_bits(u1, u2, Y, 1), want_mode(~u1, ~u2, 32, 3), "fast32_eq5 edge 1-z", u1, u2);
    }
  }
  // medium32_eq5: every small u1 class with random u2, and u2 near the low-word boundary of Z
  for (int it = 0; it < 400000; ++it) {
    const uint32_t u1 = 2u + (uint32_t)(rng() % ((1u << 22) - 1u));
    uint32_t u2 = (uint32_t)rng();
    if (it & 1) {  // Z = 4 u2 + 10 A near k 2^32
      const int64_t target = ((int64_t)(1 + rng() % 3) << 32) - (int64_t)(rng() % 24);
      const int64_t num = target - 10 * ((int64_t)u1 - 1);
      if (num < 0 || (num & 3) || num / 4 > 0xFFFFFFFFll) continue;
      u2 = (uint32_t)(num / 4);
    }
    if (!medium32_eq5_ok(u1, u2)) continue;
    const uint64_t Y = fast32_eq5_Y(u1, u2);
    expect(medium32_eq5_bits(u1, u2, Y, 0), want_mode(u1, u2, 32, 1), "medium32_eq5", u1, u2);
    expect(medium32_eq5_bits(u1, u2, Y, 1), want_mode(~u1, ~u2, 32, 3), "medium32_eq5 1-z", u1, u2);
  }
  // fast24_eq5 near the low-word boundary of K5 = (2^25 + 4) u2 + (2^26 + 10) A: solve for u2
  // modulo 2^30 ((2^23 + 1) is odd) and keep the solutions below 2^24
  for (int it = 0; it < 4000000; ++it) {
    const uint32_t u1 = 0x4001u + (uint32_t)(rng() % 0xFFB000u);
    const uint64_t A = u1 - 1u;
    const int64_t dd = -80 + (int64_t)(rng() % 88);
    const uint32_t target = (uint32_t)((int64_t)0x100000000ll + dd);
    const uint32_t rest = target - (uint32_t)(((uint64_t)1 << 26) * A + 10u * A);
    if (rest & 3u) continue;
    uint32_t inv = 1u;  // inverse of 2^23 + 1 modulo 2^30 by Newton iteration
    for (int j = 0; j < 5; ++j) inv *= 2u - ((1u << 23) + 1u) * inv;
    const uint32_t u2 = ((rest >> 2) * inv) & ((1u << 30) - 1u);
    if (u2 > 0xFFFFFFu) continue;
    const uint64_t K = fast24_eq5_K(u1, u2);
    if (!fast24_eq5_ok(u1, K)) continue;
    expect(fast24_eq5_bits(u1, u2, K, 0), want_mode(u1, u2, 24, 1), "fast24_eq5 edge", u1, u2);
    expect(fast24_eq5_bits(u1, u2, K, 0x10000u), want_mode(0xFFFFFFu - u1, 0xFFFFFFu - u2, 24, 3),
           "fast24_eq5 edge 1-z", u1, u2);
  }
  // medium24_eq5: every small u1 class with random u2, and u2 placing the low 45 bits of
  // G = m (2^24 + 2^22 + 3) next to 2^45 (checked where the medium path accepts)
  for (int it = 0; it < 400000; ++it) {
    const uint32_t u1 = 2u + (uint32_t)(rng() % 0x3FFFu);
    uint32_t u2 = (uint32_t)(rng() & 0xFFFFFFu);
    if (it & 1) {  // the u2 whose G mod 2^45 first reaches 2^45 - 2^20 - d on a random wrap j
      const uint64_t c = 0x1400003ull, base = (((uint64_t)(u1 - 1u) << 24) * c) & 0x1FFFFFFFFFFFull;
      const uint64_t t = (uint64_t)(rng() % 11) * (1ull << 45) + 0x1FFFFFF00000ull - (1u + rng() % (1u << 21));
      if (t < base) continue;
      const uint64_t v = (t - base + c - 1) / c;
      if (v > 0xFFFFFFu) continue;
      u2 = (uint32_t)v;
    }
    if (!medium24_eq5_ok(u1, u2)) continue;
    expect(medium24_eq5_bits(u1, u2, 0), want_mode(u1, u2, 24, 1), "medium24_eq5", u1, u2);
    expect(medium24_eq5_bits(u1, u2, 1), want_mode(0xFFFFFFu - u1, 0xFFFFFFu - u2, 24, 3), "medium24_eq5 1-z", u1, u2);
  }
  printf("checked %ld bad %ld\n", checked, bad);
  return bad != 0;
}
