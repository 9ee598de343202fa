// prngd_fill.cuh -- the fill kernels: one xorshift128 stream per thread, state in registers,
// outputs produced in order (Algorithm 1 per output, pair semantics for rejects), staged per
// warp in shared memory and written with 2D TMA tiled stores (cp.async.bulk.tensor) or, when
// the output cannot be described by a tensor map, with coalesced scalar stores.
#pragma once
#include <cuda.h>
#include <stdint.h>

#include "prngd_math.cuh"

namespace prngd {

constexpr int kChunk = 16;         // outputs per stream per staged tile (128 bytes per row)
constexpr int kTileBytes = 32 * kChunk * 8;  // one warp: 32 streams x 16 outputs x 8 bytes

enum Form : int { kFormA = 0, kFormB = 1, kFormC = 2 };

struct FillParams {
  uint4* state;         // n_streams xorshift states (x, y, z, w)
  uint64_t n_streams;
  uint64_t per_stream;
  uint64_t* out;        // stream-major, 8 bytes per output
  uint64_t* rejects;    // nullable, per stream
  DivConst dc;          // exact-division constants of D
  double scale;         // C_w = RN(1/D) for form A
  int w;                // draw precision
  uint32_t one;         // always 1; a run-time multiplier keeps the adds below on the FMA pipe
};

// ------------------------------------------------------------------------ per-output work
// The slow path of one output: redraw rejected pairs in order, then convert exactly. Only
// entered for a reject (probability 2^(1-w)), for small values (probability ~2^-10) and for
// the rare values near a rounding boundary of the fast paths.
template <int W, int FORM>
__device__ __forceinline__ uint64_t slow_output(uint32_t u1, uint32_t u2, XorShift128& st, uint32_t& rej,
                                                const FillParams& p) {
  const uint32_t top = (p.w == 32) ? 0xFFFFFFFFu : ((1u << p.w) - 1u);
  while (!accepted(u1, top)) {
    ++rej;
    u1 = draw<W>(st, p.w);
    u2 = draw<W>(st, p.w);
  }
  const uint64_t n = numerator(u1, u2, p.w);
  if (FORM == kFormA) return (uint64_t)__double_as_longlong(__dmul_rn(__ull2double_rn(n), p.scale));
  uint64_t bits;
  if constexpr (W == 32 || W == 24) {
    bits = rn_bits_exact(n, divconst_for<W>());
  } else {
    bits = rn_bits_exact(n, p.dc);
  }
  return FORM == kFormC ? f32pair_from_bits(bits) : bits;
}

// One output of a stream, in order. Returns the 8 output bytes.
template <int W, int FORM>
__device__ __forceinline__ uint64_t next_output(XorShift128& st, uint32_t& rej, const FillParams& p) {
  const uint32_t u1 = draw<W>(st, p.w);
  const uint32_t u2 = draw<W>(st, p.w);
  if (FORM == kFormA) {
    const uint32_t top = (W == 32) ? 0xFFFFFFFFu : (W > 0 ? ((1u << W) - 1u) : ((1u << p.w) - 1u));
    if (__builtin_expect(accepted(u1, top), 1)) {
      const int w = W > 0 ? W : p.w;
      const uint64_t n = numerator(u1, u2, w);
      return (uint64_t)__double_as_longlong(__dmul_rn(__ull2double_rn(n), p.scale));
    }
    return slow_output<W, FORM>(u1, u2, st, rej, p);
  }
  uint64_t bits;
  if (W == 32) {
    const uint64_t X = fast32_X(u1, u2);
    if (__builtin_expect(fast32_ok(u1, X), 1)) {
      bits = fast32_bits(u1, u2, X);
    } else {
      return slow_output<W, FORM>(u1, u2, st, rej, p);
    }
  } else if (W == 24) {
    const uint64_t K = fast24_K(u1, u2);
    if (__builtin_expect(fast24_ok(u1, K), 1)) {
      bits = fast24_bits(u1, u2, K);
    } else {
      return slow_output<W, FORM>(u1, u2, st, rej, p);
    }
  } else {
    return slow_output<W, FORM>(u1, u2, st, rej, p);
  }
  return FORM == kFormC ? f32pair_from_bits(bits) : bits;
}

// ------------------------------------------------------------------------ pair fast path
// Four consecutive draws in place: each state word is replaced once, so after the block
// (x, y, z, w) is again the state in its usual order and the four draws are its words.
__device__ __forceinline__ uint32_t xs_word(uint32_t a, uint32_t w) {
  const uint32_t t = a ^ (a << 11);
  return w ^ (w >> 19) ^ (t ^ (t >> 8));
}
__device__ __forceinline__ void xs_block4(XorShift128& s) {
  s.x = xs_word(s.x, s.w);
  s.y = xs_word(s.y, s.x);
  s.z = xs_word(s.z, s.y);
  s.w = xs_word(s.w, s.z);
}

// The w = 32 form-B fast path of fast32_ok / fast32_bits written out as PTX, with the adds
// that need no carry issued as multiply-adds by the run-time constant `one` so that they run
// on the FMA pipe beside the ALU work of the draws. Returns 1 in `ok` when the fast path
// applies (same condition as fast32_ok); the value is meaningless otherwise.
__device__ __forceinline__ uint64_t fast32_bits_ptx(uint32_t u1, uint32_t u2, uint32_t one, uint32_t& ok) {
  uint32_t lo, hi;
  asm("{\n\t"
      ".reg .u64 Y, X, P, Ip;\n\t"
      ".reg .u32 xlo, f, a, A, g, ilo, ihi, q, s, rb, jlo, jhi, s1, mhi, e;\n\t"
      ".reg .pred p1, p2;\n\t"
      "mad.wide.u32 Y, %4, 2, -1;\n\t"           // 2 u2 - 1
      "mad.wide.u32 X, %3, 3, Y;\n\t"            // X = 2B + 3A = 3 u1 + 2 u2 - 1
      "mov.b64 {xlo, f}, X;\n\t"
      "mad.lo.u32 a, %3, %5, -4194305;\n\t"      // u1 - (2^22 + 1)
      "setp.lt.u32 p1, a, 0xFFBFFFFD;\n\t"       // 2^22 <= A <= 2^32 - 4
      "setp.lt.and.u32 p2, xlo, 0xFFFFFFF8, p1;\n\t"
      "selp.u32 %1, 1, 0, p2;\n\t"
      "mad.lo.u32 A, %3, %5, -1;\n\t"            // A = u1 - 1
      "mov.b64 P, {%4, A};\n\t"
      "mad.wide.u32 Ip, A, 2, P;\n\t"            // A 2^32 + u2 + 2A
      "mad.lo.u32 g, f, %5, 1;\n\t"
      "mov.b64 {ilo, ihi}, Ip;\n\t"
      "add.cc.u32 ilo, ilo, g;\n\t"              // I = A 2^32 + B + 2A + (X >> 32)
      "addc.u32 ihi, ihi, 0;\n\t"
      "bfind.u32 q, ihi;\n\t"                    // p, top bit of the high word
      "mad.lo.u32 s, q, %5, -21;\n\t"
      "shl.b32 rb, 1, s;\n\t"
      "add.cc.u32 jlo, ilo, rb;\n\t"             // J = I + 2^s
      "addc.u32 jhi, ihi, 0;\n\t"
      "mad.lo.u32 s1, q, %5, -20;\n\t"
      "shf.r.wrap.b32 %2, jlo, jhi, s1;\n\t"     // mantissa, low word
      "shr.u32 mhi, jhi, s1;\n\t"
      "mad.lo.u32 e, q, 0x100000, 0x3DE00000;\n\t"  // (p + 990) << 20
      "mad.lo.u32 %0, mhi, %5, e;\n\t"
      "}"
      : "=r"(hi), "=r"(ok), "=r"(lo)
      : "r"(u1), "r"(u2), "r"(one));
  return ((uint64_t)hi << 32) | lo;
}

struct PairOut {
  uint64_t v0, v1;
  uint32_t x, y, z, w, rej;
};

// Exact replay of two outputs (w = 32 or 24). (x, y, z, w) is the state after the pair's 4-draw
// block; it is rewound 4 steps to the block's start, then the two outputs are redrawn with
// in-order rejects and converted exactly.
template <int FORM, int W>
__device__ __noinline__ PairOut slow_pair(uint32_t x, uint32_t y, uint32_t z, uint32_t w, uint32_t rej) {
  constexpr int wbits = W;
  const DivConst dc = divconst_for<W>();
  XorShift128 st{x, y, z, w};
  xs_prev(st);
  xs_prev(st);
  xs_prev(st);
  xs_prev(st);
  const uint32_t top = (wbits == 32) ? 0xFFFFFFFFu : ((1u << wbits) - 1u);
  uint64_t v[2];
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    uint32_t u1 = draw<0>(st, wbits), u2 = draw<0>(st, wbits);
    while (!accepted(u1, top)) {
      ++rej;
      u1 = draw<0>(st, wbits);
      u2 = draw<0>(st, wbits);
    }
    const uint64_t bits = rn_bits_exact(numerator(u1, u2, wbits), dc);
    v[k] = FORM == kFormC ? f32pair_from_bits(bits) : bits;
  }
  return PairOut{v[0], v[1], st.x, st.y, st.z, st.w, rej};
}

// Two outputs of a w = 32 or w = 24 stream (forms B and C) from one 4-draw block, with one
// branch for the pair. A small value takes the inline medium path; a reject or a value near
// a rounding boundary replays the pair exactly from the block's starting state.
template <int W, int FORM>
__device__ __forceinline__ void next_pair(XorShift128& st, uint32_t& rej, const FillParams& p, uint64_t& v0,
                                          uint64_t& v1) {
  xs_block4(st);
  uint32_t ok;
  if constexpr (W == 32) {
    uint32_t ok0, ok1;
    v0 = fast32_bits_ptx(st.x, st.y, p.one, ok0);
    v1 = fast32_bits_ptx(st.z, st.w, p.one, ok1);
    ok = ok0 & ok1;
  } else {
    const uint32_t u1a = st.x >> 8, u2a = st.y >> 8, u1b = st.z >> 8, u2b = st.w >> 8;
    const uint64_t Ka = fast24_K(u1a, u2a), Kb = fast24_K(u1b, u2b);
    ok = fast24_ok(u1a, Ka) & fast24_ok(u1b, Kb);
    v0 = fast24_bits(u1a, u2a, Ka);
    v1 = fast24_bits(u1b, u2b, Kb);
  }
  if (__builtin_expect(ok == 0, 0)) {
    // Almost always a small value (A < 2^22 at w = 32): the inline medium path. Rejects and
    // values near a rounding boundary replay the pair exactly.
    bool replay = false;
    if constexpr (W == 32) {
      const uint64_t Xa = fast32_X(st.x, st.y), Xb = fast32_X(st.z, st.w);
      if (!fast32_ok(st.x, Xa)) {
        if (medium32_ok(st.x, Xa, st.y)) v0 = medium32_bits(st.x, st.y, Xa); else replay = true;
      }
      if (!fast32_ok(st.z, Xb)) {
        if (medium32_ok(st.z, Xb, st.w)) v1 = medium32_bits(st.z, st.w, Xb); else replay = true;
      }
    } else {
      const uint32_t u1a = st.x >> 8, u2a = st.y >> 8, u1b = st.z >> 8, u2b = st.w >> 8;
      const uint64_t Ka = fast24_K(u1a, u2a), Kb = fast24_K(u1b, u2b);
      if (!fast24_ok(u1a, Ka)) {
        if (medium24_ok(u1a, Ka, u2a)) v0 = medium24_bits(u1a, u2a, Ka); else replay = true;
      }
      if (!fast24_ok(u1b, Kb)) {
        if (medium24_ok(u1b, Kb, u2b)) v1 = medium24_bits(u1b, u2b, Kb); else replay = true;
      }
    }
    if (replay) {
      const PairOut o = slow_pair<kFormB, W>(st.x, st.y, st.z, st.w, rej);
      v0 = o.v0;
      v1 = o.v1;
      rej = o.rej;
      st = XorShift128{o.x, o.y, o.z, o.w};
    }
  }
  if (FORM == kFormC) {
    v0 = f32pair_from_bits(v0);
    v1 = f32pair_from_bits(v1);
  }
}

// ------------------------------------------------------------------------ PTX helpers
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void fence_async_shared() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void tma_store_2d(const CUtensorMap* map, uint32_t src, int x, int y) {
  asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%2, %3}], [%1];" ::"l"(map),
               "r"(src), "r"(x), "r"(y)
               : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void bulk_wait_read() {
  asm volatile("cp.async.bulk.wait_group.read %0;" ::"n"(N) : "memory");
}
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void st_shared_v2(uint32_t addr, uint64_t a, uint64_t b) {
  asm volatile("st.shared.v2.b64 [%0], {%1, %2};" ::"r"(addr), "l"(a), "l"(b) : "memory");
}

// ------------------------------------------------------------------------ kernels
// TMA path. Warp g owns streams 32g .. 32g+31 (lane = row of the tile). Per chunk of 16
// outputs each lane computes its 16 outputs in registers, writes them as 8 x 16-byte pieces
// into the warp's tile with the 128-byte swizzle (piece c of row r at r*128 + ((c ^ (r & 7))
// * 16)), and lane 0 issues one 2D bulk tensor store of the 32 x 16 box. Rows past n_streams
// and columns past per_stream fall outside the tensor and are not written. NBUF tiles per
// warp let the next chunk's staging proceed while the previous store still reads shared memory.
template <int W, int FORM, int NBUF>
__global__ void __launch_bounds__(256, 4) fill_tma_kernel(const FillParams p,
                                                       const __grid_constant__ CUtensorMap tmap) {
  extern __shared__ uint8_t smem_raw[];
  const uint32_t base = (smem_addr(smem_raw) + 1023u) & ~1023u;
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const uint64_t warp_global = (uint64_t)blockIdx.x * (blockDim.x >> 5) + warp;
  if (warp_global * 32 >= p.n_streams) return;  // the whole warp is past the last stream
  const uint64_t stream = warp_global * 32 + lane;
  const bool active = stream < p.n_streams;
  uint4 s4 = active ? p.state[stream] : make_uint4(1u, 2u, 3u, 4u);
  XorShift128 st{s4.x, s4.y, s4.z, s4.w};
  uint32_t rej = 0;
  const uint32_t tile0 = base + (uint32_t)warp * NBUF * kTileBytes;
  const uint32_t row_off = (uint32_t)lane * 128u;
  const uint32_t sw = (uint32_t)(lane & 7);
  const int y0 = (int)(warp_global * 32);
  uint32_t chunk_idx = 0;
  for (uint64_t x0 = 0; x0 < p.per_stream; x0 += kChunk, ++chunk_idx) {
    uint64_t v[kChunk];
    const uint64_t left = p.per_stream - x0;
    if (left >= (uint64_t)kChunk) {
      if constexpr ((W == 32 || W == 24) && FORM != kFormA) {
#pragma unroll
        for (int j = 0; j < kChunk; j += 2) next_pair<W, FORM>(st, rej, p, v[j], v[j + 1]);
      } else {
#pragma unroll
        for (int j = 0; j < kChunk; ++j) v[j] = next_output<W, FORM>(st, rej, p);
      }
    } else {
#pragma unroll
      for (int j = 0; j < kChunk; ++j) v[j] = (j < (int)left) ? next_output<W, FORM>(st, rej, p) : 0ull;
    }
    const uint32_t tile = tile0 + (chunk_idx % NBUF) * kTileBytes;
    if (lane == 0) bulk_wait_read<NBUF - 1>();
    __syncwarp();
#pragma unroll
    for (int c = 0; c < kChunk / 2; ++c)
      st_shared_v2(tile + row_off + (((uint32_t)c ^ sw) << 4), v[2 * c], v[2 * c + 1]);
    fence_async_shared();
    __syncwarp();
    if (lane == 0) {
      tma_store_2d(&tmap, tile, (int)x0, y0);
      bulk_commit();
    }
  }
  if (lane == 0) bulk_wait_all();
  if (active) {
    p.state[stream] = make_uint4(st.x, st.y, st.z, st.w);
    if (p.rejects) p.rejects[stream] = rej;
  }
}

// Generic store path (any alignment, any per_stream): the warp stages its 32 x 16 tile with a
// padded row pitch of 17 words and writes it back row by row, 16 lanes per row, so each store
// instruction covers two 128-byte row segments.
template <int W, int FORM>
__global__ void __launch_bounds__(256) fill_plain_kernel(const FillParams p) {
  __shared__ uint64_t tiles[8][32 * (kChunk + 1)];
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const uint64_t warp_global = (uint64_t)blockIdx.x * (blockDim.x >> 5) + warp;
  const uint64_t stream = warp_global * 32 + lane;
  const bool active = stream < p.n_streams;
  uint4 s4 = active ? p.state[stream] : make_uint4(1u, 2u, 3u, 4u);
  XorShift128 st{s4.x, s4.y, s4.z, s4.w};
  uint32_t rej = 0;
  uint64_t* tile = tiles[warp];
  for (uint64_t x0 = 0; x0 < p.per_stream; x0 += kChunk) {
    const uint64_t left = p.per_stream - x0;
    const int cnt = left >= (uint64_t)kChunk ? kChunk : (int)left;
#pragma unroll
    for (int j = 0; j < kChunk; ++j)
      if (j < cnt) tile[lane * (kChunk + 1) + j] = next_output<W, FORM>(st, rej, p);
    __syncwarp();
#pragma unroll
    for (int i = 0; i < kChunk; ++i) {
      const int idx = i * 32 + lane;
      const int row = idx / kChunk, col = idx % kChunk;
      const uint64_t s = warp_global * 32 + row;
      if (col < cnt && s < p.n_streams) p.out[s * p.per_stream + x0 + col] = tile[row * (kChunk + 1) + col];
    }
    __syncwarp();
  }
  if (active) {
    p.state[stream] = make_uint4(st.x, st.y, st.z, st.w);
    if (p.rejects) p.rejects[stream] = rej;
  }
}

}  // namespace prngd
