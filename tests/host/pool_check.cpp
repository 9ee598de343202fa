// Host check of the serving loop's output-pool allocator (prngd_pool.h) against a plain model:
// one flag per 256-byte granule. Random allocations and releases; after every operation the
// allocator's answer must be the first-fit answer of the model (the lowest maximal free run
// that holds the request, or none), its free ranges must be exactly the model's maximal free
// runs (so free neighbours were merged), and its byte count in use must match. Built and run
// by test_host_pool.py. Prints "bad <count>" and exits non-zero on any mismatch.
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <random>
#include <utility>
#include <vector>

#include "prngd_pool.h"

using prngd_host::RangePool;

namespace {

constexpr size_t G = RangePool::kGranule;

struct Model {
  std::vector<uint8_t> busy;
  explicit Model(size_t granules) : busy(granules, 0) {}
  // maximal free runs as (first granule, length)
  std::vector<std::pair<size_t, size_t>> runs() const {
    std::vector<std::pair<size_t, size_t>> r;
    for (size_t i = 0; i < busy.size();) {
      if (busy[i]) {
        ++i;
        continue;
      }
      size_t j = i;
      while (j < busy.size() && !busy[j]) ++j;
      r.push_back({i, j - i});
      i = j;
    }
    return r;
  }
  size_t first_fit(size_t k) const {
    for (auto& run : runs())
      if (run.second >= k) return run.first;
    return SIZE_MAX;
  }
  void mark(size_t first, size_t k, uint8_t v) {
    for (size_t i = first; i < first + k; ++i) busy[i] = v;
  }
  size_t used() const {
    size_t n = 0;
    for (uint8_t b : busy) n += b;
    return n;
  }
};

long bad = 0;

void check_state(const RangePool& pool, const Model& m, long step) {
  std::vector<std::pair<size_t, size_t>> got;
  pool.for_each_free([&](size_t off, size_t len) { got.push_back({off / G, len / G}); });
  if (got != m.runs()) {
    if (bad < 5) printf("step %ld: free ranges differ from the model's maximal runs\n", step);
    ++bad;
  }
  if (pool.used() != m.used() * G) {
    if (bad < 5) printf("step %ld: used %zu, model %zu\n", step, pool.used(), m.used() * G);
    ++bad;
  }
}

void run(uint64_t seed, size_t pool_bytes, size_t max_bytes, long ops) {
  std::mt19937_64 rng(seed);
  RangePool pool(pool_bytes);
  Model m(pool_bytes / G);
  std::vector<std::pair<size_t, size_t>> live;  // (offset, requested bytes)
  for (long step = 0; step < ops; ++step) {
    const bool do_alloc = live.empty() || (rng() % 100) < 55;
    if (do_alloc) {
      // log-uniform sizes in [1, max_bytes], with exact granule multiples and 0 mixed in
      size_t bytes;
      const unsigned kind = rng() % 10;
      if (kind == 0) {
        bytes = 0;
      } else if (kind == 1) {
        bytes = G * (1 + rng() % (max_bytes / G));
      } else {
        const double u = std::uniform_real_distribution<double>(0.0, 1.0)(rng);
        bytes = (size_t)std::exp(u * std::log((double)max_bytes));
      }
      const size_t k = RangePool::footprint(bytes) / G;
      const size_t want = m.first_fit(k);
      const size_t off = pool.alloc(bytes);
      const size_t got = off == RangePool::kNone ? SIZE_MAX : off / G;
      if (got != want || (off != RangePool::kNone && off % G)) {
        if (bad < 5) printf("step %ld: alloc(%zu) gave %zu, first fit %zu\n", step, bytes, got, want);
        ++bad;
      }
      if (off != RangePool::kNone && got == want) {
        m.mark(got, k, 1);
        live.push_back({off, bytes});
      }
    } else {
      const size_t i = rng() % live.size();
      const auto a = live[i];
      live[i] = live.back();
      live.pop_back();
      pool.release(a.first, a.second);
      m.mark(a.first / G, RangePool::footprint(a.second) / G, 0);
    }
    check_state(pool, m, step);
  }
  // release everything: one free range of the whole pool
  for (const auto& a : live) {
    pool.release(a.first, a.second);
    m.mark(a.first / G, RangePool::footprint(a.second) / G, 0);
  }
  check_state(pool, m, ops);
  if (pool.free_ranges() != 1 || pool.used() != 0) {
    printf("after releasing everything: %zu free ranges, %zu bytes used\n", pool.free_ranges(), pool.used());
    ++bad;
  }
  // a request larger than the pool never fits
  if (pool.alloc(pool_bytes + 1) != RangePool::kNone) {
    printf("alloc larger than the pool succeeded\n");
    ++bad;
  }
}

}  // namespace

int main() {
  run(1, 1 << 20, 64 << 10, 20000);   // many small requests: fragmentation, merging
  run(2, 1 << 20, 1 << 20, 20000);    // requests up to the whole pool: frequent refusals
  run(3, 3 * G, 3 * G, 2000);         // a pool of three granules
  run(4, (1 << 16) + 100, 1 << 14, 5000);  // a size that is not a granule multiple
  printf("bad %ld\n", bad);
  return bad ? 1 : 0;
}
