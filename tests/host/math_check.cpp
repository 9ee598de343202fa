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

int main() {
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
  printf("checked %ld bad %ld\n", checked, bad);
  return bad != 0;
}
