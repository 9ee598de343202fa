// prngd_jump.cu -- jump-ahead for the xorshift128 streams and the split fill.
//
// xorshift128 is linear over GF(2): one step is a 128 x 128 matrix T acting on the state, so
// the state after J draws is T^J s. With P the characteristic polynomial of T (degree 128,
// found here by Berlekamp-Massey from one output bit) and g = x^J mod P, Cayley-Hamilton
// gives T^J = g(T), so T^J s = sum_i g_i T^i s: 128 steps and up to 128 xors of states.
//
// The split fill uses this to cut each stream into S segments of `seg` attempts. With the pair
// rule (Section 2: a rejected pair is dropped whole) attempt a always uses draws 2a and 2a + 1,
// so segment j starts at the state T^(2 j seg) s whatever happened before it, and its accepted
// attempts are outputs j seg - R_j, ... of the stream, R_j the rejects before it. The main
// pass runs the fill kernel over the segments as if each were a stream of `seg` outputs: that
// is exact for every segment with no reject in it or before it. Rejects are rare (2/2^w per
// attempt), so the streams that had one are repaired by small kernels: recount the nominal
// rejects of the affected segments, prefix-sum them, regenerate those segments at their
// shifted positions, and draw the stream's missing last outputs after its last segment.
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <mutex>
#include <vector>

#include "prngd_fill.cuh"
#include "prngd_gf2.h"
#include "prngd_internal.h"

namespace prngd {

constexpr int kMaxSplitLog2 = 23;  // at most 2^23 segments per stream
// Segment index in base 8192: one jump for up to 8192 segments per stream, two beyond (the
// table holds 128 KiB per digit; base 256 took two jumps at 8192 segments, 8% of a split fill).
constexpr int kJumpDigitBits = 13;
constexpr uint32_t kJumpBase = 1u << kJumpDigitBits;
constexpr int kJumpDigits = 2;  // 26 bits >= kMaxSplitLog2

// T^(delta j) s from a table of jump polynomials over the base-8192 digits of j:
// table[d * 8192 + k] = x^(delta k 8192^d) mod P (k = 0 entries unused).
__device__ __forceinline__ XorShift128 jump_to_segment(const uint4* __restrict__ table, uint32_t j, XorShift128 st) {
#pragma unroll 1
  for (int d = 0; d < kJumpDigits; ++d) {
    const uint32_t k = (j >> (kJumpDigitBits * d)) & (kJumpBase - 1u);
    if (k) {
      const uint4 q = table[d * kJumpBase + k];
      const uint32_t g[4] = {q.x, q.y, q.z, q.w};
      st = apply_poly(g, st);
    }
  }
  return st;
}

// Start state of every segment row (row = s S + j): T^(delta j) applied to stream s's state.
// Segment 0 of each stream also resets the stream's first-bad marker to S.
__global__ void jump_rows_kernel(const uint4* __restrict__ base, uint4* __restrict__ rows, uint64_t n_rows,
                                 int log2s, const uint4* __restrict__ table, uint32_t* __restrict__ first_bad) {
  const uint64_t row = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (row >= n_rows) return;
  const uint64_t s = row >> log2s;
  const uint32_t j = (uint32_t)(row & ((1ull << log2s) - 1));
  if (j == 0) first_bad[s] = 1u << log2s;
  const uint4 b4 = base[s];
  const XorShift128 st = jump_to_segment(table, j, XorShift128{b4.x, b4.y, b4.z, b4.w});
  rows[row] = make_uint4(st.x, st.y, st.z, st.w);
}

// The same for 2^8 or more segments per stream, where a block's 256 rows lie in one stream and
// share the high base-8192 digit k1 of their segment index j = k0 + 8192 k1. With
// u = T^(delta 8192 k1) s, T^(delta j) s = T^(delta k0) u = sum_i g_i T^i u with
// g = x^(delta k0) mod P, and the 128 states T^i u are the same for every row of the block:
// one thread makes u (a jump from the state) and steps the powers into shared memory, the
// block tabulates the xor of every subset of each 4 consecutive powers, and each row is then 32
// table entries (one per 4 coefficients of g) xored together, with no generator steps (a jump
// from the state alone also steps the generator 128 times). Measured on the 2^20 rows of 64
// streams x 16384 segments: 117 us from the state, 57 us from shared powers by 128 masked xors
// (the ALU pipe's load), about 14 us less with the 4-coefficient table (the split call 639 ->
// 644 Gsamples/s in one harness); making the powers once per group in a separate kernel saved
// no more than the masked xors did (55 us).
// u = T^(delta 8192 k1) s: the block's high digit, once per block, out of line so that its
// registers do not count against the row loop's occupancy.
__device__ __noinline__ XorShift128 jump_high_digit(const uint4* __restrict__ table, uint32_t k1, XorShift128 st) {
  const uint4 q = table[kJumpBase + k1];
  const uint32_t g[4] = {q.x, q.y, q.z, q.w};
  return apply_poly(g, st);
}

__global__ void __launch_bounds__(256) jump_rows_shared_kernel(const uint4* __restrict__ base, uint4* __restrict__ rows,
                                                                uint64_t n_rows, int log2s,
                                                                const uint4* __restrict__ table,
                                                                uint32_t* __restrict__ first_bad) {
  __shared__ uint4 powers[128];  // T^i u, i = 0 .. 127
  const uint64_t row0 = (uint64_t)blockIdx.x * blockDim.x;
  const uint64_t s = row0 >> log2s;
  const uint64_t seg_mask = (1ull << log2s) - 1;
  if (threadIdx.x == 0) {
    const uint4 b4 = base[s];
    XorShift128 st{b4.x, b4.y, b4.z, b4.w};
    const uint32_t k1 = (uint32_t)((row0 & seg_mask) >> kJumpDigitBits);  // the block's high digit
    if (k1) st = jump_high_digit(table, k1, st);
    for (int i = 0; i < 128; ++i) {
      powers[i] = make_uint4(st.x, st.y, st.z, st.w);
      xs_next(st);
    }
  }
  __syncthreads();
  // The xor of every subset of each four consecutive powers (32 groups x 16 subsets), so that a
  // row takes one table entry per 4 coefficients: 32 loads and xors instead of 128 masked ones.
  __shared__ uint4 combo[32 * 16];
  for (uint32_t e = threadIdx.x; e < 32 * 16; e += blockDim.x) {
    const uint32_t grp = e >> 4, c = e & 15u;
    uint4 acc = make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      if ((c >> b) & 1u) {
        const uint4 v = powers[4 * grp + b];
        acc.x ^= v.x;
        acc.y ^= v.y;
        acc.z ^= v.z;
        acc.w ^= v.w;
      }
    }
    combo[e] = acc;
  }
  __syncthreads();
  const uint64_t row = row0 + threadIdx.x;
  if (row >= n_rows) return;
  const uint32_t j = (uint32_t)(row & seg_mask);
  if (j == 0) first_bad[s] = 1u << log2s;  // segment 0 also resets the stream's first-bad marker
  const uint32_t k0 = j & (kJumpBase - 1u);
  if (k0 == 0) {  // T^0 u
    rows[row] = powers[0];
    return;
  }
  const uint4 q = table[k0];
  const uint32_t g[4] = {q.x, q.y, q.z, q.w};
  uint32_t ax = 0, ay = 0, az = 0, aw = 0;
#pragma unroll
  for (int word = 0; word < 4; ++word) {
#pragma unroll
    for (int nib = 0; nib < 8; ++nib) {
      const uint4 v = combo[16 * (8 * word + nib) + ((g[word] >> (4 * nib)) & 15u)];
      ax ^= v.x;
      ay ^= v.y;
      az ^= v.z;
      aw ^= v.w;
    }
  }
  rows[row] = make_uint4(ax, ay, az, aw);
}

// Every stream advanced by J draws: state <- g(T) state, g = x^J mod P.
__global__ void skip_kernel(uint4* __restrict__ state, uint64_t n, const uint4 g4) {
  const uint64_t s = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (s >= n) return;
  const uint32_t g[4] = {g4.x, g4.y, g4.z, g4.w};
  const uint4 v = state[s];
  const XorShift128 st = apply_poly(g, XorShift128{v.x, v.y, v.z, v.w});
  state[s] = make_uint4(st.x, st.y, st.z, st.w);
}

struct SplitArgs {
  const uint4* base;     // the streams' states before the call
  uint4* rows;           // per segment row: after the main pass its end state; repaired rows: start state
  const uint64_t* rej;   // per segment row: rejects the main pass met (any nonzero marks the stream)
  uint32_t* nom;         // per segment row: rejects in its nominal attempts (affected streams)
  uint32_t* first_bad;   // per stream: the first segment with a reject (S if none)
  uint32_t* total;       // per stream: all nominal rejects R_S
  uint4* tail;           // per stream: the state after its last segment's nominal attempts
  uint64_t n_streams;
  uint32_t log2s;
  uint64_t seg;          // attempts (outputs) per segment
  const uint4* table;    // jump polynomials over the base-8192 digits of the segment index
};

// Per segment row: a row whose main pass met a reject lowers its stream's first-bad marker.
__global__ void split_first_bad_kernel(const SplitArgs a) {
  const uint64_t row = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (row >= (a.n_streams << a.log2s)) return;
  if (a.rej[row] != 0) atomicMin(a.first_bad + (row >> a.log2s), (uint32_t)(row & ((1ull << a.log2s) - 1)));
}

// Affected streams, segments from the first bad one on: the start state again (jump), kept in
// rows[], and the rejects among the segment's own attempts; the last segment also leaves the
// state after its attempts for the tail.
template <int W>
__global__ void split_count_kernel(const SplitArgs a, int w) {
  const uint64_t row = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  const uint64_t n_rows = a.n_streams << a.log2s;
  if (row >= n_rows) return;
  const uint64_t s = row >> a.log2s;
  const uint32_t j = (uint32_t)(row & ((1ull << a.log2s) - 1));
  if (j < a.first_bad[s]) {
    a.nom[row] = 0;
    return;
  }
  const uint4 b4 = a.base[s];
  XorShift128 st = jump_to_segment(a.table, j, XorShift128{b4.x, b4.y, b4.z, b4.w});
  a.rows[row] = make_uint4(st.x, st.y, st.z, st.w);
  const uint32_t top = (w == 32) ? 0xFFFFFFFFu : ((1u << w) - 1u);
  uint32_t r = 0;
  for (uint64_t k = 0; k < a.seg; ++k) {
    const uint32_t u1 = draw<W>(st, w);
    draw<W>(st, w);
    r += accepted(u1, top) ? 0u : 1u;
  }
  a.nom[row] = r;
  if (j == (1u << a.log2s) - 1u) a.tail[s] = make_uint4(st.x, st.y, st.z, st.w);
}

// One warp per affected stream: the exclusive prefix sum of the nominal rejects over its
// segments (in place) and their total.
__global__ void split_scan_kernel(const SplitArgs a) {
  const uint64_t s = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (s >= a.n_streams) return;
  const uint32_t S = 1u << a.log2s;
  const uint32_t first = a.first_bad[s];
  uint32_t carry = 0;
  if (first < S) {
    for (uint32_t j0 = first & ~31u; j0 < S; j0 += 32) {
      const uint32_t j = j0 + lane;
      const uint32_t v = (j < S) ? a.nom[(s << a.log2s) + j] : 0u;
      uint32_t incl = v;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const uint32_t o = __shfl_up_sync(0xffffffffu, incl, d);
        if (lane >= d) incl += o;
      }
      if (j < S) a.nom[(s << a.log2s) + j] = carry + incl - v;  // rejects before segment j
      carry += __shfl_sync(0xffffffffu, incl, 31);
    }
  }
  if (lane == 0) a.total[s] = carry;
}

// Affected segments: their accepted attempts, exactly converted, at the stream's true output
// positions j seg - R_j + k.
template <int W, int FORM, int MAP>
__global__ void split_regen_kernel(const SplitArgs a, const FillParams p) {
  const uint64_t row = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  const uint64_t n_rows = a.n_streams << a.log2s;
  if (row >= n_rows) return;
  const uint64_t s = row >> a.log2s;
  const uint32_t j = (uint32_t)(row & ((1ull << a.log2s) - 1));
  if (j < a.first_bad[s]) return;
  const uint4 b4 = a.rows[row];
  XorShift128 st{b4.x, b4.y, b4.z, b4.w};
  const uint32_t top = (p.w == 32) ? 0xFFFFFFFFu : ((1u << p.w) - 1u);
  const uint64_t per = a.seg << a.log2s;
  uint64_t* dst = p.out + s * per + (uint64_t)j * a.seg - a.nom[row];
  uint64_t k = 0;
  for (uint64_t i = 0; i < a.seg; ++i) {
    const uint32_t u1 = draw<W>(st, p.w);
    const uint32_t u2 = draw<W>(st, p.w);
    if (!accepted(u1, top)) continue;
    dst[k++] = convert_accepted<W, FORM, MAP>(u1, u2, p);
  }
}

// Per stream: the outputs still missing after the last segment (one per nominal reject), drawn
// in order after it; the stream's final state and its reject count.
template <int FORM, int MAP>
__global__ void split_tail_kernel(const SplitArgs a, const FillParams p, uint4* __restrict__ state,
                                  uint64_t* __restrict__ rejects) {
  const uint64_t s = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (s >= a.n_streams) return;
  const uint32_t S = 1u << a.log2s;
  if (a.first_bad[s] == S) {  // no reject anywhere: the main pass's last end state is final
    state[s] = a.rows[(s << a.log2s) + S - 1];
    if (rejects) rejects[s] = 0;
    return;
  }
  const uint4 t4 = a.tail[s];
  XorShift128 st{t4.x, t4.y, t4.z, t4.w};
  const uint32_t missing = a.total[s];
  const uint64_t per = a.seg << a.log2s;
  uint32_t rej = 0;
  for (uint32_t k = 0; k < missing; ++k)
    p.out[s * per + per - missing + k] = next_output<0, FORM, MAP>(st, rej, p);
  state[s] = make_uint4(st.x, st.y, st.z, st.w);
  if (rejects) rejects[s] = (uint64_t)missing + rej;
}

}  // namespace prngd

namespace prngd_host {
namespace {

Poly g_charpoly;
bool g_charpoly_ok = false;
std::once_flag g_charpoly_once;

bool charpoly_ready() {
  std::call_once(g_charpoly_once, [] { g_charpoly_ok = find_charpoly(&g_charpoly); });
  return g_charpoly_ok;
}
Poly x_pow(uint64_t J) { return x_pow_mod(J, g_charpoly); }
Poly mulmod(const Poly& a, const Poly& b) { return mulmod_p(a, b, g_charpoly); }

template <int FORM, int MAP>
cudaError_t launch_repair(const prngd::SplitArgs& a, const prngd::FillParams& p, uint4* state, uint64_t* rejects,
                          cudaStream_t s) {
  const uint64_t n_rows = a.n_streams << a.log2s;
  const unsigned rb = (unsigned)((n_rows + 255) / 256), sb = (unsigned)((a.n_streams + 255) / 256);
  if (p.w == 32 && (FORM == prngd::kFormB || FORM == prngd::kFormC))
    prngd::split_regen_kernel<32, FORM, MAP><<<rb, 256, 0, s>>>(a, p);
  else
    prngd::split_regen_kernel<0, FORM, MAP><<<rb, 256, 0, s>>>(a, p);
  prngd::split_tail_kernel<FORM, MAP><<<sb, 256, 0, s>>>(a, p, state, rejects);
  return cudaGetLastError();
}

template <int FORM>
cudaError_t launch_repair_map(int map, const prngd::SplitArgs& a, const prngd::FillParams& p, uint4* state,
                              uint64_t* rejects, cudaStream_t s) {
  switch (map) {
    case 0: return launch_repair<FORM, 0>(a, p, state, rejects, s);
    case prngd::kMapEq5: return launch_repair<FORM, prngd::kMapEq5>(a, p, state, rejects, s);
    case prngd::kMapOneMinus: return launch_repair<FORM, prngd::kMapOneMinus>(a, p, state, rejects, s);
    default: return launch_repair<FORM, prngd::kMapEq5 | prngd::kMapOneMinus>(a, p, state, rejects, s);
  }
}

}  // namespace

void release_split(prng_ctx* h) {
  if (h->split_mem) cudaFree(h->split_mem);
  h->split_mem = nullptr;
  h->split_bytes = 0;
  h->split_table_seg = 0;
  h->split_table_mem = nullptr;
  h->split_table_digits = 0;
}

int skip_streams(prng_ctx* h, uint64_t draws, cudaStream_t s) {
  if (!charpoly_ready()) return fail(PRNG_ECUDA, "jump polynomial: characteristic polynomial not found");
  if (draws == 0) return PRNG_OK;
  uint32_t g[4];
  words_of(x_pow(draws), g);
  prngd::skip_kernel<<<(unsigned)((h->n_streams + 255) / 256), 256, 0, s>>>(h->d_state, h->n_streams,
                                                                        make_uint4(g[0], g[1], g[2], g[3]));
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(PRNG_ECUDA, "skip launch: %s", cudaGetErrorString(e));
  return PRNG_OK;
}

// Segments per stream when the caller leaves it to the library: the smallest power of two that
// gives about four rows per thread slot of the GPU, keeping segments of at least 1024 outputs.
uint32_t auto_segments(prng_ctx* h, uint64_t per_stream) {
  const uint64_t target = (uint64_t)h->num_sms * 2048 * 4;
  uint32_t S = 1;
  while ((uint64_t)h->n_streams * S < target && S < (1u << prngd::kMaxSplitLog2) && per_stream % (2ull * S) == 0 &&
         per_stream / (2ull * S) >= 1024)
    S *= 2;
  return S;
}

int fill_split(prng_ctx* h, void* out, uint64_t per_stream, int form, int mode, uint32_t segments,
               uint64_t* rejects, cudaStream_t s) {
  if (mode & PRNG_MODE_SINGLE_REDRAW)
    return fail(PRNG_EINVAL, "the split fill needs the pair reject rule (Algorithm 1's single redraw has no "
                             "fixed attempt boundaries)");
  if (segments == 0) segments = auto_segments(h, per_stream);
  if ((segments & (segments - 1)) || segments > (1u << prngd::kMaxSplitLog2) || per_stream % segments)
    return fail(PRNG_EINVAL, "segments must be a power of two (<= 2^23) dividing per_stream");
  if (segments == 1)
    return launch_fill(h, h->d_state, h->n_streams, out, per_stream, form, rejects, s, true, mode);
  if (!charpoly_ready()) return fail(PRNG_ECUDA, "jump polynomial: characteristic polynomial not found");
  int log2s = 0;
  while ((1u << log2s) < segments) ++log2s;
  const uint64_t seg = per_stream / segments;
  const uint64_t n_rows = h->n_streams << log2s;
  // scratch: the jump table first (a fixed place, so a later call never overwrites it), then per
  // row the state (16 B), the main-pass rejects (8 B) and the nominal rejects (4 B), then per
  // stream the tail state (16 B), the first bad segment and the total (4 B each)
  const size_t table_bytes = (size_t)prngd::kJumpDigits * prngd::kJumpBase * 16;
  const size_t bytes = table_bytes + n_rows * 28 + h->n_streams * 24 + 256;
  if (h->split_bytes < bytes) {
    release_split(h);
    cudaError_t e = cudaMalloc(&h->split_mem, bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(PRNG_ENOMEM, "split scratch (%zu bytes): %s", bytes, cudaGetErrorString(e));
    }
    h->split_bytes = bytes;
  }
  char* base = (char*)h->split_mem;
  uint4* table = (uint4*)base;
  char* rest = base + table_bytes;
  uint4* rows = (uint4*)rest;
  uint64_t* rej = (uint64_t*)(rest + n_rows * 16);
  uint32_t* nom = (uint32_t*)(rest + n_rows * 24);
  uint4* tail = (uint4*)(rest + ((n_rows * 28 + 15) & ~(size_t)15));
  uint32_t* first_bad = (uint32_t*)(tail + h->n_streams);
  uint32_t* total = first_bad + h->n_streams;

  prngd::SplitArgs a;
  a.base = h->d_state;
  a.rows = rows;
  a.rej = rej;
  a.nom = nom;
  a.first_bad = first_bad;
  a.total = total;
  a.tail = tail;
  a.n_streams = h->n_streams;
  a.log2s = (uint32_t)log2s;
  a.seg = seg;
  a.table = table;
  const int digits = (log2s + prngd::kJumpDigitBits - 1) / prngd::kJumpDigitBits;  // digits j can have
  if (h->split_table_seg != seg || h->split_table_mem != (void*)table || h->split_table_digits < digits) {
    // x^(delta k 8192^d) mod P for the digits segment indices use, k < 8192, delta = 2 seg draws
    // (pair rule); built on the host once per segment length (a few ms a digit) and copied to
    // the start of the scratch
    static thread_local std::vector<uint4> host;
    host.assign((size_t)digits * prngd::kJumpBase, make_uint4(0, 0, 0, 0));
    Poly step = x_pow(2 * seg);
    for (int d = 0; d < digits; ++d) {
      Poly acc{1, 0};
      for (uint32_t k = 1; k < prngd::kJumpBase; ++k) {
        acc = mulmod(acc, step);
        uint32_t g[4];
        words_of(acc, g);
        host[(size_t)d * prngd::kJumpBase + k] = make_uint4(g[0], g[1], g[2], g[3]);
      }
      step = mulmod(acc, step);  // x^(delta 8192^(d+1))
    }
    cudaError_t ce = cudaMemcpyAsync(table, host.data(), host.size() * sizeof(uint4), cudaMemcpyHostToDevice, s);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);  // `host` is reused by the next call
    if (ce != cudaSuccess) return fail(PRNG_ECUDA, "jump table copy: %s", cudaGetErrorString(ce));
    h->split_table_seg = seg;
    h->split_table_mem = table;
    h->split_table_digits = digits;
  }
  const unsigned rb = (unsigned)((n_rows + 255) / 256);
  if (log2s >= 8) {  // a block's 256 rows in one stream, sharing the high digit
    prngd::jump_rows_shared_kernel<<<rb, 256, 0, s>>>(h->d_state, rows, n_rows, log2s, table, first_bad);
  } else {
    prngd::jump_rows_kernel<<<rb, 256, 0, s>>>(h->d_state, rows, n_rows, log2s, table, first_bad);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(PRNG_ECUDA, "jump launch: %s", cudaGetErrorString(e));
  // main pass: every segment as a stream of `seg` outputs
  int rc = launch_fill(h, rows, n_rows, out, seg, form, rej, s, true, mode);
  if (rc) return rc;
  // repair of the streams that met a reject
  const unsigned wb = (unsigned)((h->n_streams * 32 + 255) / 256);
  prngd::split_first_bad_kernel<<<rb, 256, 0, s>>>(a);
  if (h->w == 32)
    prngd::split_count_kernel<32><<<rb, 256, 0, s>>>(a, h->w);
  else
    prngd::split_count_kernel<0><<<rb, 256, 0, s>>>(a, h->w);
  prngd::split_scan_kernel<<<wb, 256, 0, s>>>(a);
  prngd::FillParams p;
  memset(&p, 0, sizeof(p));
  p.out = (uint64_t*)out;
  p.dc = h->dc;
  p.scale = h->scale;
  p.w = h->w;
  p.one = 1;
  set_mode_constants(p, h->w, mode);
  const int map = mode & (PRNG_MODE_EQ5 | PRNG_MODE_ONE_MINUS);
  switch (form) {
    case PRNG_FORM_A_FP64: e = launch_repair_map<prngd::kFormA>(map, a, p, h->d_state, rejects, s); break;
    case PRNG_FORM_C_F32PAIR: e = launch_repair_map<prngd::kFormC>(map, a, p, h->d_state, rejects, s); break;
    case PRNG_FORM_L_ALGO1: e = launch_repair_map<prngd::kFormL>(map, a, p, h->d_state, rejects, s); break;
    default: e = launch_repair_map<prngd::kFormB>(map, a, p, h->d_state, rejects, s); break;
  }
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) return fail(PRNG_ECUDA, "split repair launch: %s", cudaGetErrorString(e));
  return PRNG_OK;
}

}  // namespace prngd_host

using namespace prngd_host;

extern "C" {

int prng_skip(prng_t h, uint64_t draws, void* cuda_stream) {
  if (!h) return fail(PRNG_EINVAL, "null handle");
  int rc = require_xorshift(h, "prng_skip");
  if (!rc) rc = check_handle_device(h);
  if (rc) return rc;
  return skip_streams(h, draws, (cudaStream_t)cuda_stream);
}

int prng_fill_split(prng_t h, void* d_out, uint64_t per_stream, int form, int mode, uint32_t segments,
                    uint64_t* d_rejects, void* cuda_stream) {
  if (!h) return fail(PRNG_EINVAL, "null handle");
  if (form != PRNG_FORM_A_FP64 && form != PRNG_FORM_B_INTBITS && form != PRNG_FORM_C_F32PAIR &&
      form != PRNG_FORM_L_ALGO1)
    return fail(PRNG_EINVAL, "unknown form %d", form);
  if (mode & ~kAllModes) return fail(PRNG_EINVAL, "unknown mode bits 0x%x", (unsigned)mode);
  if (per_stream == 0) return PRNG_OK;
  if (!d_out) return fail(PRNG_EINVAL, "d_out is NULL");
  if ((uintptr_t)d_out & 7) return fail(PRNG_EINVAL, "d_out must be 8-byte aligned");
  int rc = require_xorshift(h, "prng_fill_split");
  if (!rc) rc = check_fill_extent(h, per_stream, d_rejects);
  if (!rc) rc = check_handle_device(h);
  if (rc) return rc;
  return fill_split(h, d_out, per_stream, form, mode, segments, d_rejects, (cudaStream_t)cuda_stream);
}

}  // extern "C"
