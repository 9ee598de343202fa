// Host-compiled check of the library's MRG32k3a step (prngd_mrg.cuh) against the oracle: long
// runs from seeded states and single steps from states at the edges of both moduli. Built and
// run by test_host_mrg.py.
#include <cstdint>
#include <cstdio>
#include <random>

#include "prngd_mrg.cuh"

extern "C" {
uint32_t orc_mrg32k3a_next(uint32_t st[6]);
void orc_mrg_stream_seed(uint64_t seed, uint64_t stream, uint32_t st[6]);
}

using namespace prngd;

int main() {
  long bad = 0, checked = 0;
  auto run = [&](uint32_t st[6], int steps) {
    Mrg32k3a g{st[0], st[1], st[2], st[3], st[4], st[5]};
    for (int i = 0; i < steps; ++i) {
      const uint32_t want = orc_mrg32k3a_next(st);
      const uint32_t got = mrg_next(g);
      ++checked;
      if (got != want || g.a0 != st[0] || g.a1 != st[1] || g.a2 != st[2] || g.b0 != st[3] || g.b1 != st[4] ||
          g.b2 != st[5]) {
        if (bad < 10) printf("mismatch: got %u want %u\n", got, want);
        ++bad;
        return;
      }
    }
  };
  for (uint64_t s = 0; s < 64; ++s) {
    uint32_t st[6];
    orc_mrg_stream_seed(12345, s, st);
    run(st, 20000);
  }
  std::mt19937_64 rng(3);
  const uint32_t m1 = 4294967087u, m2 = 4294944443u;
  const uint32_t e1[6] = {0u, 1u, 2u, m1 - 1u, m1 - 2u, m1 / 2u}, e2[6] = {0u, 1u, 2u, m2 - 1u, m2 - 2u, m2 / 2u};
  for (int i = 0; i < 200000; ++i) {
    uint32_t st[6];
    for (int k = 0; k < 3; ++k) {
      st[k] = (i & 1) ? e1[rng() % 6] : (uint32_t)(rng() % m1);
      st[3 + k] = (i & 2) ? e2[rng() % 6] : (uint32_t)(rng() % m2);
    }
    run(st, 3);
  }
  // the reductions against %, for v < 2^54: random, and at multiples of 2^32, m1 and m2 +- small
  auto check_mod = [&](uint64_t v) {
    if (v >> 54) return;  // outside the reductions' domain (k = 0, d < 0 wraps)
    ++checked;
    if (mod_m1(v) != (uint32_t)(v % m1) || mod_m2(v) != (uint32_t)(v % m2)) {
      if (bad < 10) printf("mod mismatch v=%llu\n", (unsigned long long)v);
      ++bad;
    }
  };
  for (int i = 0; i < 4000000; ++i) check_mod(rng() >> 10);
  for (uint64_t k = 0; k < (1ull << 22); k += 1 + (k >> 6))
    for (int d = -3; d <= 3; ++d) {
      check_mod((k << 32) + (uint64_t)(int64_t)d);
      check_mod(k * m1 + (uint64_t)(int64_t)d);
      check_mod(k * m2 + (uint64_t)(int64_t)d);
    }
  check_mod((1ull << 54) - 1);
  // the conversion's fast path: floor(n 2^64 / D) exactly wherever it reports ok, on random n,
  // on n of each binade's ends, and on n placing the low word of S next to 2^32
  const unsigned __int128 D = (unsigned __int128)(m1 - 1u) * (m1 - 1u);
  auto check_fast = [&](uint64_t n) {
    if (n == 0 || (unsigned __int128)n >= D) return;
    uint32_t ok;
    const uint64_t I = mrg_fast_I(n, ok);
    if (!ok) return;
    ++checked;
    const uint64_t want = (uint64_t)(((unsigned __int128)n << 64) / D);
    if (I != want) {
      if (bad < 10) printf("mrg_fast_I mismatch n=%llu\n", (unsigned long long)n);
      ++bad;
    }
  };
  for (int i = 0; i < 4000000; ++i) check_fast(rng() % (uint64_t)((m1 - 1ull) * (m1 - 1ull)));
  for (int p = 54; p < 64; ++p)
    for (int d = -64; d < 64; ++d) check_fast((1ull << p) + (uint64_t)(int64_t)d);
  long near = 0;
  for (int i = 0; i < 400000; ++i) {  // nl solving 420 nl = k 2^32 - (132300 nh mod 2^32) - d: S's low
    const uint64_t nh = rng() % (m1 - 2u);       // word lands within a few hundred of 2^32
    const uint64_t k = 1 + rng() % 419, d = rng() % 600;
    uint64_t nl = 0;
    for (int it = 0; it < 2; ++it) {  // the carry term (E2 >> 32) depends on nl: refine once
      const uint64_t e = (132300u * nl + 37044000u * nh) >> 32;
      const int64_t num = (int64_t)((k << 32) - ((132300u * nh + e) & 0xFFFFFFFFull)) - (int64_t)d;
      nl = num < 0 ? (1ull << 40) : (uint64_t)num / 420u;
    }
    if (nl > 0xFFFFFFFFull) continue;
    const uint64_t n = (nh << 32) | nl;
    const uint64_t S = 420u * nl + 132300u * nh + ((132300u * nl + 37044000u * nh) >> 32);
    if ((uint32_t)S >= 0xFFFFF000u) ++near;
    check_fast(n);
  }
  printf("near-margin samples %ld\n", near);
  printf("checked %ld bad %ld\n", checked, bad);
  return bad != 0;
}
