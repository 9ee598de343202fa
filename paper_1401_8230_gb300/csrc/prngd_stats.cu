// prngd_stats.cu -- host entry point of the fused statistics kernel.
#include <cuda_runtime.h>
#include <stdint.h>

#include "prngd.h"
#include "prngd_internal.h"
#include "prngd_launch.h"
#include "prngd_stats.cuh"

namespace prngd_host {

static constexpr uint32_t kMaxStatsBlock = 992;  // T * kStatsInterval must stay <= 32767
static constexpr size_t kStatsSmem = (size_t)prngd::kHistWords * 4;

// Block size T (a multiple of 32, <= 992) such that the streams fill whole rounds of one
// block per SM: rounds = ceil(n / (SMs * 992)), T = ceil(n / (SMs * rounds)) rounded up to 32.
uint32_t stats_block_size(uint64_t n_streams, int num_sms) {
  const uint64_t per_round = (uint64_t)num_sms * kMaxStatsBlock;
  const uint64_t rounds = (n_streams + per_round - 1) / per_round;
  uint64_t t = (n_streams + (uint64_t)num_sms * rounds - 1) / ((uint64_t)num_sms * rounds);
  t = (t + 31) / 32 * 32;
  if (t < 32) t = 32;
  if (t > kMaxStatsBlock) t = kMaxStatsBlock;
  return (uint32_t)t;
}

template <int W>
static cudaError_t launch_stats_w(const prngd::StatsParams& p, int num_sms, cudaStream_t s) {
  auto k = prngd::stats_kernel<W>;
  static std::atomic<uint64_t> attr{0};
  const cudaError_t e = prngd::smem_limit_once(k, (int)kStatsSmem, attr);
  if (e != cudaSuccess) return e;
  const uint64_t units = (p.n_streams + p.unit - 1) / p.unit;
  const unsigned grid = (unsigned)(units < (uint64_t)num_sms ? units : (uint64_t)num_sms);
  k<<<grid, p.unit, kStatsSmem, s>>>(p);
  return cudaGetLastError();
}

int launch_stats(prng_ctx* h, uint64_t per_stream, uint64_t* d_hist, uint64_t* d_sums, uint64_t* d_rejects,
                 cudaStream_t s) {
  prngd::StatsParams p;
  p.state = h->d_state;
  p.n_streams = h->n_streams;
  p.per_stream = per_stream;
  p.hist = d_hist;
  p.sums = d_sums;
  p.rejects = d_rejects;
  p.dc = h->dc;
  p.w = h->w;
  p.unit = stats_block_size(h->n_streams, h->num_sms);
  p.one = 1;
  cudaError_t e;
  if (h->w == 32)
    e = launch_stats_w<32>(p, h->num_sms, s);
  else if (h->w == 24)
    e = launch_stats_w<24>(p, h->num_sms, s);
  else
    e = launch_stats_w<0>(p, h->num_sms, s);
  if (e != cudaSuccess) return fail(PRNG_ECUDA, "stats launch: %s", cudaGetErrorString(e));
  return PRNG_OK;
}

}  // namespace prngd_host

using namespace prngd_host;

extern "C" int prng_stats_merge(const uint64_t* hist_in, const uint64_t* sums_in, uint64_t* hist_acc,
                                uint64_t* sums_acc) {
  if (!hist_in || !sums_in || !hist_acc || !sums_acc) return fail(PRNG_EINVAL, "null pointer");
  for (int i = 0; i < 2 * prngd::kHistWords; ++i) hist_acc[i] += hist_in[i];
  for (int p = 0; p < 4; ++p) {
    const uint64_t lo = sums_acc[2 * p] + sums_in[2 * p];
    sums_acc[2 * p + 1] += sums_in[2 * p + 1] + (lo < sums_in[2 * p] ? 1u : 0u);
    sums_acc[2 * p] = lo;
  }
  return PRNG_OK;
}

extern "C" int prng_fused_stats(prng_t h, uint64_t per_stream, uint64_t* d_hist, uint64_t* d_sums,
                                uint64_t* d_rejects, void* cuda_stream) {
  if (!h) return fail(PRNG_EINVAL, "null handle");
  if (!d_hist || !d_sums) return fail(PRNG_EINVAL, "d_hist and d_sums are required");
  if (((uintptr_t)d_hist & 7) || ((uintptr_t)d_sums & 7)) return fail(PRNG_EINVAL, "d_hist/d_sums must be 8-byte aligned");
  if (per_stream == 0) return PRNG_OK;
  int rc = require_xorshift(h, "prng_fused_stats");
  if (!rc) rc = check_fill_extent(h, per_stream, d_rejects);
  if (!rc) rc = check_handle_device(h);
  if (rc) return rc;
  return launch_stats(h, per_stream, d_hist, d_sums, d_rejects, (cudaStream_t)cuda_stream);
}
