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
  const unsigned __int128 D = (unsigned __int128)(m1 - 1u) * (m1 - 1u);
  // the conversion's fast path from A = u1 - 1 and B = u2 + 1: floor(n 2^64 / D) exactly wherever
  // it reports ok, on random pairs, at the ends of both ranges, and on B placing the low word of
  // S next to 2^32
  const uint64_t M = m1;
  long near_ab = 0, refused_ab = 0;
  auto check_ab = [&](uint64_t A, uint64_t B) {
    if (A < (1u << 22) || A > M - 3 || B < 1 || B > M) return;
    uint32_t ok;
    const uint64_t I = mrg_fast_I_ab((uint32_t)A, (uint32_t)B, ok);
    if (!ok) {
      ++refused_ab;
      return;
    }
    ++checked;
    const uint64_t want = (uint64_t)(((unsigned __int128)(A * M + B) << 64) / D);
    if (I != want) {
      if (bad < 10) printf("mrg_fast_I_ab mismatch A=%llu B=%llu\n", (unsigned long long)A, (unsigned long long)B);
      ++bad;
    }
  };
  for (int i = 0; i < 4000000; ++i) check_ab((1u << 22) + rng() % (M - 2 - (1u << 22)), 1 + rng() % M);
  for (uint64_t A : {(uint64_t)1 << 22, ((uint64_t)1 << 22) + 1, M / 2, M - 4, M - 3})
    for (uint64_t B : {(uint64_t)1, (uint64_t)2, M / 2, M - 1, M}) check_ab(A, B);
  for (int i = 0; i < 400000; ++i) {  // B solving 44520 A + 420 B + (W >> 32) = k 2^32 - d
    const uint64_t A = (1u << 22) + rng() % (M - 2 - (1u << 22));
    const uint64_t d = rng() % 600;
    uint64_t B = 1 + rng() % M;
    for (int it = 0; it < 2; ++it) {  // (W >> 32) depends on B: refine once
      const uint64_t wh = (9393300u * A + 132300u * B) >> 32;
      const uint64_t base = 44520u * A + wh;
      const uint64_t T = ((base + 420u * B) >> 32 << 32) + (1ull << 32) - d;  // the next boundary, minus d
      B = (T - base) / 420u;
    }
    const uint64_t wh = (9393300u * A + 132300u * B) >> 32;
    const uint64_t S = 44520u * A + 420u * B + wh;
    if ((uint32_t)S >= 0xFFFFF000u) ++near_ab;
    check_ab(A, B);
  }
  printf("near-margin samples (A, B) %ld refused %ld\n", near_ab, refused_ab);
  printf("checked %ld bad %ld\n", checked, bad);
  return bad != 0;
}
