// prngd_stats.cuh -- fused statistics without storing values: the streams advance exactly as
// in a fill, and each output contributes to a 65536-bin histogram of floor(2^16 z') and to
// the integer moment sums of t = floor(2^32 z'), p2 = floor(t^2/2^32), p3 = floor(p2 t/2^32),
// p4 = floor(p3 t/2^32). z' = n/D exactly, so every result is an exact integer.
#pragma once
#include <stdint.h>

#include "prngd_math.cuh"

namespace prngd {

struct StatsParams {
  uint4* state;
  uint64_t n_streams;
  uint64_t per_stream;
  uint64_t* hist;     // 65536 counters, accumulated
  uint64_t* sums;     // S1..S4 as 128-bit (lo, hi) pairs, accumulated
  uint64_t* rejects;  // nullable
  DivConst dc;
  int w;
  uint32_t unit;      // streams per work unit (= block size)
  uint32_t one;       // 1, read at run time (multiply-adds by it stay on the FMA pipe)
};

constexpr int kHistWords = 32768;  // word i holds bin i (low half) and bin i + 32768 (high half)
constexpr int kStatsInterval = 32; // outputs per thread between overflow checks (T * 32 <= 32767)

// floor(V 2^64) exactly, by one 2-by-1 division of (n 2^sh) 2^64 by D' = D 2^sh.
PRNGD_HD uint64_t floor_v64_exact(uint64_t n, const DivConst& dc) {
  const uint64_t u1 = n << dc.sh;  // < D'
  uint64_t q0 = dc.v * u1;
  uint64_t q1 = umulhi64(dc.v, u1);
  q1 += u1;  // + (u1, u0) with u0 = 0
  q1 += 1;
  uint64_t r = 0 - q1 * dc.d_norm;
  if (r > q0) {
    q1 -= 1;
    r += dc.d_norm;
  }
  if (r >= dc.d_norm) q1 += 1;
  return q1;
}

// t = floor(2^32 V) of the next output of a stream (in order, rejects redrawn as pairs).
template <int W>
__device__ __forceinline__ uint32_t next_t(XorShift128& st, uint32_t& rej, const StatsParams& p) {
  uint32_t u1 = draw<W>(st, p.w);
  uint32_t u2 = draw<W>(st, p.w);
  if constexpr (W == 32) {
    // floor(V 2^64) = A 2^32 + (B + 2A) + (X >> 32) when the low word of X is not within 8 of
    // 2^32 (see fast32_bits); its high word is t.
    // As the fill's PTX: 3 u1 + 2 u2 = X + 1 by a wide multiply and multiply-add (no 64-bit
    // constant), X's low word by one 32-bit multiply-add, then A 2^32 + 2A + u2 + (X >> 32) + 1
    // with the carry into the high word, which is t (measured at 2^36 outputs: 549 -> 586
    // Gsamples/s against the same sums in C, which carried the -1 as a 64-bit constant).
    uint32_t t, ok;
    asm("{\n\t"
        ".reg .u64 Y, X, P, J;\n\t"
        ".reg .u32 xlo, f, A, g, jlo, jhi;\n\t"
        ".reg .pred p1, p2;\n\t"
        "mul.wide.u32 Y, %3, 2;\n\t"
        "mad.wide.u32 X, %2, 3, Y;\n\t"
        "mov.b64 {xlo, f}, X;\n\t"
        "mad.lo.u32 xlo, xlo, %4, -1;\n\t"
        "mad.lo.u32 A, %2, %4, -1;\n\t"
        "setp.lt.u32 p1, A, 0xFFFFFFFE;\n\t"
        "setp.lt.and.u32 p2, xlo, 0xFFFFFFF8, p1;\n\t"
        "selp.u32 %1, 1, 0, p2;\n\t"
        "mov.b64 P, {%3, A};\n\t"
        "mad.wide.u32 J, A, 2, P;\n\t"
        "mad.lo.u32 g, f, %4, 1;\n\t"
        "mov.b64 {jlo, jhi}, J;\n\t"
        "add.cc.u32 jlo, jlo, g;\n\t"
        "addc.u32 %0, jhi, 0;\n\t"
        "}"
        : "=r"(t), "=r"(ok)
        : "r"(u1), "r"(u2), "r"(p.one));
    if (__builtin_expect(ok != 0, 1)) return t;
  } else if constexpr (W == 24) {
    const uint64_t K = fast24_K(u1, u2);
    if (__builtin_expect((((uint32_t)(u1 - 1u) < 0xFFFFFEu) & ((uint32_t)K < 0xFFFFFFF0u)) != 0, 1)) {
      const uint32_t A = u1 - 1u, B = u2 + 1u;
      const uint64_t low = ((uint64_t)(B + 2u * A) << 16) + (K >> 32);
      return (A << 8) + (uint32_t)(low >> 32);
    }
  }
  const uint32_t top = (p.w == 32) ? 0xFFFFFFFFu : ((1u << p.w) - 1u);
  while (!accepted(u1, top)) {
    ++rej;
    u1 = draw<W>(st, p.w);
    u2 = draw<W>(st, p.w);
  }
  return (uint32_t)(floor_v64_exact(numerator(u1, u2, p.w), p.dc) >> 32);
}

__device__ __forceinline__ void add_u128_shared(unsigned long long* lo, unsigned long long* hi, uint64_t v) {
  if (!v) return;
  const unsigned long long old = atomicAdd(lo, (unsigned long long)v);
  if (old + v < old) atomicAdd(hi, 1ull);
}

__device__ __forceinline__ void add_u128_global(uint64_t* lohi, uint64_t lo, uint64_t hi) {
  const unsigned long long old = atomicAdd((unsigned long long*)&lohi[0], (unsigned long long)lo);
  if (old + lo < old) ++hi;
  if (hi) atomicAdd((unsigned long long*)&lohi[1], (unsigned long long)hi);
}

// Persistent kernel: block b processes work units b, b + gridDim.x, ...; unit u is streams
// [u*T, (u+1)*T) with T = blockDim.x, one stream per thread. The histogram lives in shared
// memory as 16-bit counters; a counter is at most 2^15 at the start of an interval (an
// increment that returns a half >= 2^15 asks for a flush, decided by the OR over the block
// at the interval's barrier) and gains at most T * kStatsInterval <= 32767 within it, so it never wraps.
template <int W>
__global__ void __launch_bounds__(1024, 1) stats_kernel(const StatsParams p) {
  extern __shared__ uint32_t hist[];
  __shared__ unsigned long long s_sum[8];
  const uint32_t T = blockDim.x;
  for (uint32_t i = threadIdx.x; i < kHistWords; i += T) hist[i] = 0;
  if (threadIdx.x < 8) s_sum[threadIdx.x] = 0;
  __syncthreads();

  const uint64_t n_units = (p.n_streams + p.unit - 1) / p.unit;
  for (uint64_t u = blockIdx.x; u < n_units; u += gridDim.x) {
    const uint64_t stream = u * p.unit + threadIdx.x;
    const bool active = stream < p.n_streams;
    uint4 s4 = active ? p.state[stream] : make_uint4(1u, 2u, 3u, 4u);
    XorShift128 st{s4.x, s4.y, s4.z, s4.w};
    uint32_t rej = 0;
    uint64_t a1 = 0, a2 = 0, a3 = 0, a4 = 0;
    uint64_t since_fold = 0;
    for (uint64_t x0 = 0; x0 < p.per_stream; x0 += kStatsInterval) {
      const uint64_t left = p.per_stream - x0;
      const int cnt = left >= (uint64_t)kStatsInterval ? kStatsInterval : (int)left;
      uint32_t ovf = 0;
      if (active) {
#pragma unroll 8
        for (int j = 0; j < cnt; ++j) {
          const uint32_t t = next_t<W>(st, rej, p);
          // bin = t >> 16; low half for bins < 32768, high half for the rest
          const uint32_t inc = (t >> 31) * 0xFFFFu + 1u;
          ovf |= atomicAdd(&hist[(t >> 16) & 0x7FFFu], inc);
          const uint64_t tt = (uint64_t)t * t;
          const uint32_t p2 = (uint32_t)(tt >> 32);
          const uint32_t p3 = (uint32_t)(((uint64_t)p2 * t) >> 32);
          const uint32_t p4 = (uint32_t)(((uint64_t)p3 * t) >> 32);
          a1 += t;
          a2 += p2;
          a3 += p3;
          a4 += p4;
        }
      }
      since_fold += cnt;
      // The barrier's OR gives every thread the same answer, so the flush branch (and the
      // barrier inside it) is taken by the whole block or by none of it.
      if (__syncthreads_or((ovf & 0x80008000u) != 0u)) {
        for (uint32_t i = threadIdx.x; i < kHistWords; i += T) {
          const uint32_t v = hist[i];
          hist[i] = 0;
          if (v & 0xFFFFu) atomicAdd((unsigned long long*)&p.hist[i], (unsigned long long)(v & 0xFFFFu));
          if (v >> 16) atomicAdd((unsigned long long*)&p.hist[i + 32768], (unsigned long long)(v >> 16));
        }
        __syncthreads();  // the next interval's increments start on the zeroed counters
      }
      if (since_fold >= (1ull << 24)) {  // per-thread 64-bit sums hold < 2^24 terms of < 2^32
        add_u128_shared(&s_sum[0], &s_sum[1], a1);
        add_u128_shared(&s_sum[2], &s_sum[3], a2);
        add_u128_shared(&s_sum[4], &s_sum[5], a3);
        add_u128_shared(&s_sum[6], &s_sum[7], a4);
        a1 = a2 = a3 = a4 = 0;
        since_fold = 0;
      }
    }
    add_u128_shared(&s_sum[0], &s_sum[1], a1);
    add_u128_shared(&s_sum[2], &s_sum[3], a2);
    add_u128_shared(&s_sum[4], &s_sum[5], a3);
    add_u128_shared(&s_sum[6], &s_sum[7], a4);
    if (active) {
      p.state[stream] = make_uint4(st.x, st.y, st.z, st.w);
      if (p.rejects) p.rejects[stream] = rej;
    }
  }
  __syncthreads();
  for (uint32_t i = threadIdx.x; i < kHistWords; i += T) {
    const uint32_t v = hist[i];
    if (v & 0xFFFFu) atomicAdd((unsigned long long*)&p.hist[i], (unsigned long long)(v & 0xFFFFu));
    if (v >> 16) atomicAdd((unsigned long long*)&p.hist[i + 32768], (unsigned long long)(v >> 16));
  }
  if (threadIdx.x < 4) add_u128_global(&p.sums[2 * threadIdx.x], s_sum[2 * threadIdx.x], s_sum[2 * threadIdx.x + 1]);
}

}  // namespace prngd
