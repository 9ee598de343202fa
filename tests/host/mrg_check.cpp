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
  printf("checked %ld bad %ld\n", checked, bad);
  return bad != 0;
}
