// prngd_mrg.cu -- streams of L'Ecuyer's MRG32k3a (Operations Research 47(1), 1999), one of the
// base generators Section 2 recommends, and the fill over them.
//
// Two order-3 recurrences, x1_n = (1403580 x1_{n-2} - 810728 x1_{n-3}) mod m1 and
// x2_n = (527612 x2_{n-1} - 1370589 x2_{n-3}) mod m2 with m1 = 2^32 - 209, m2 = 2^32 - 22853,
// combined as z = (x1 - x2) mod m1 in [1, m1] (0 reported as m1). The method reads z as the
// draw u = z - 1 on a grid of M = m1 points with step k = 1/M, so Section 2 holds with 2^w
// replaced by M: pairs with u1 in {0, M - 1} are rejected and z' = n / D with
// n = u1 M + u2 - (M - 1), D = (M - 1)^2 < 2^64, converted by a series fast path (mrg_fast_I_ab)
// or exactly (Moller-Granlund division) for small values and margin cases.
//
// State: 32 bytes per stream in the handle's state array (two uint4: x1_{n-3}, x1_{n-2},
// x1_{n-1}, x2_{n-3} | x2_{n-2}, x2_{n-1}, 0, 0), seeded from splitmix64 outputs 3s, 3s+1, 3s+2.
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include "prngd_fill.cuh"
#include "prngd_internal.h"
#include "prngd_launch.h"
#include "prngd_mrg.cuh"

namespace prngd {

__device__ __forceinline__ Mrg32k3a mrg_load(const uint4* state, uint64_t s) {
  const uint4 a = state[2 * s], b = state[2 * s + 1];
  return Mrg32k3a{a.x, a.y, a.z, a.w, b.x, b.y};
}
__device__ __forceinline__ void mrg_store(uint4* state, uint64_t s, const Mrg32k3a& g) {
  state[2 * s] = make_uint4(g.a0, g.a1, g.a2, g.b0);
  state[2 * s + 1] = make_uint4(g.b1, g.b2, 0u, 0u);
}

// Stream s of `seed`: splitmix64 outputs 3s, 3s+1, 3s+2 as six 32-bit words (low word first),
// reduced modulo m1 (x1 words) and m2 (x2 words); an all-zero component gets 1 as its first word.
__global__ void mrg_seed_kernel(uint4* state, uint64_t n, uint64_t seed) {
  const uint64_t s = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (s >= n) return;
  uint32_t w[6];
  for (int i = 0; i < 3; ++i) {
    const uint64_t o = splitmix_finalise(seed + (3 * s + (uint64_t)i + 1) * kGoldenGamma);
    w[2 * i] = (uint32_t)o;
    w[2 * i + 1] = (uint32_t)(o >> 32);
  }
  Mrg32k3a g{w[0] % kMrgM1, w[1] % kMrgM1, w[2] % kMrgM1, w[3] % kMrgM2, w[4] % kMrgM2, w[5] % kMrgM2};
  if ((g.a0 | g.a1 | g.a2) == 0) g.a0 = 1;
  if ((g.b0 | g.b1 | g.b2) == 0) g.b0 = 1;
  mrg_store(state, s, g);
}

#ifndef PRNGD_MRG_UNROLL
#define PRNGD_MRG_UNROLL 2
#endif
// output pairs unrolled in a chunk's loop: measured with the pair path (form B / balanced / C,
// Gsamples/s) 2: 294 / 307 / 275, 4: 293 / 305 / 274, all 8: 293 / 302 / 275
constexpr int kMrgUnroll = PRNGD_MRG_UNROLL;

// The rare cases of an output, out of line so that the unrolled chunk stays within the
// instruction cache (inline, the chunk stalled on instruction fetch: form B 260 -> 283
// Gsamples/s out of line): a rejected pair (u1 in {0, M - 1}, probability 2/M) is followed by the
// next pairs until one is accepted; small values and margin cases take the exact division.
struct MrgRedraw {
  Mrg32k3a g;
  uint32_t rej, u1, u2;
};
__device__ __noinline__ MrgRedraw mrg_redraw(Mrg32k3a g, uint32_t rej) {
  uint32_t u1, u2;
  do {
    ++rej;
    u1 = mrg_next(g) - 1u;
    u2 = mrg_next(g) - 1u;
  } while (u1 - 1u >= kMrgM1 - 2u);
  return MrgRedraw{g, rej, u1, u2};
}
__device__ __noinline__ uint64_t mrg_exact_bits(uint32_t u1, uint32_t u2, DivConst dc) {
  return rn_bits_exact((uint64_t)u1 * kMrgM1 + u2 - (kMrgM1 - 1u), dc);
}

// One output of the method over MRG32k3a draws (pair rule), 8 bytes of form FORM; MAP is 0 or
// kMapCvt (PRNG_MODE_BALANCED, form B's rounding route).
template <int FORM, int MAP = 0>
__device__ __forceinline__ uint64_t mrg_next_output(Mrg32k3a& g, uint32_t& rej, const FillParams& p) {
  // the usual case, an accepted pair, is straight-line code (no loop around the state's
  // rotation)
  uint32_t u1 = mrg_next(g) - 1u;
  uint32_t u2 = mrg_next(g) - 1u;
  if (__builtin_expect(u1 - 1u >= kMrgM1 - 2u, 0)) {
    const MrgRedraw r = mrg_redraw(g, rej);
    g = r.g;
    rej = r.rej;
    u1 = r.u1;
    u2 = r.u2;
  }
  // n = u1 M + u2 - (M - 1), formed only where it is used
  // form A: the conversion instruction, then the scale (its definition's two FP64 steps)
  if constexpr (FORM == kFormA)
    return (uint64_t)__double_as_longlong(__dmul_rn(__ull2double_rn((uint64_t)u1 * kMrgM1 + u2 - (kMrgM1 - 1u)), p.scale));
  uint64_t bits;
  uint32_t ok = 0;
  if (__builtin_expect(u1 > (1u << 22), 1)) {  // A >= 2^22: the series fast path
    const uint64_t I = mrg_fast_I_ab(u1 - 1u, u2 + 1u, ok);
    // the fills' rounding routes (cvt_group_mask): form C by the conversion instruction; form B
    // by integer operations, or by the conversion under PRNG_MODE_BALANCED (measured 283 and
    // 300 Gsamples/s)
    bits = cvt_group_mask<FORM, 32, MAP>() ? bits_from_I_cvt(I, p.one) : bits_from_I_int(I, p.one);
  }
  if (__builtin_expect(!ok, 0)) {  // small values, margin cases
    bits = mrg_exact_bits(u1, u2, p.dc);
  }
  return FORM == kFormC ? f32pair_from_bits(bits) : bits;
}

// Two outputs of a form-B or form-C stream with one check and one branch: the four draws are
// taken, both fast paths run, and if either pair was rejected, either value is small or near
// a rounding boundary, the two outputs are replayed exactly from the state before them
// (measured: form B 283 -> 294 Gsamples/s against one check per output).
struct MrgPair {
  Mrg32k3a g;
  uint32_t rej;
  uint64_t v0, v1;
};
template <int FORM, int MAP>
__device__ __noinline__ MrgPair mrg_pair_replay(Mrg32k3a g, uint32_t rej, const FillParams p);

template <int FORM, int MAP = 0>
__device__ __forceinline__ void mrg_next_pair(Mrg32k3a& g, uint32_t& rej, const FillParams& p, uint64_t& v0,
                                              uint64_t& v1) {
  const Mrg32k3a g0 = g;
  const uint32_t a1 = mrg_next(g) - 1u, a2 = mrg_next(g) - 1u;
  const uint32_t b1 = mrg_next(g) - 1u, b2 = mrg_next(g) - 1u;
  uint32_t oka, okb;
  const uint64_t Ia = mrg_fast_I_ab(a1 - 1u, a2 + 1u, oka);
  const uint64_t Ib = mrg_fast_I_ab(b1 - 1u, b2 + 1u, okb);
  // accepted (u1 - 1 < M - 2) with A >= 2^22, i.e. u1 in (2^22, M - 1), and no margin case
  const uint32_t fast = (uint32_t)(a1 - ((1u << 22) + 1u) < kMrgM1 - 1u - ((1u << 22) + 1u)) &
                        (uint32_t)(b1 - ((1u << 22) + 1u) < kMrgM1 - 1u - ((1u << 22) + 1u)) & oka & okb;
  if (__builtin_expect(fast != 0, 1)) {
    const bool cv = cvt_group_mask<FORM, 32, MAP>() != 0;
    const uint64_t ba = cv ? bits_from_I_cvt(Ia, p.one) : bits_from_I_int(Ia, p.one);
    const uint64_t bb = cv ? bits_from_I_cvt(Ib, p.one) : bits_from_I_int(Ib, p.one);
    v0 = FORM == kFormC ? f32pair_from_bits(ba) : ba;
    v1 = FORM == kFormC ? f32pair_from_bits(bb) : bb;
  } else {
    const MrgPair r = mrg_pair_replay<FORM, MAP>(g0, rej, p);
    g = r.g;
    rej = r.rej;
    v0 = r.v0;
    v1 = r.v1;
  }
}

template <int FORM, int MAP>
__device__ __noinline__ MrgPair mrg_pair_replay(Mrg32k3a g, uint32_t rej, const FillParams p) {
  const uint64_t v0 = mrg_next_output<FORM, MAP>(g, rej, p);
  const uint64_t v1 = mrg_next_output<FORM, MAP>(g, rej, p);
  return MrgPair{g, rej, v0, v1};
}

// Tile-staged TMA path with SPT streams per thread and CH outputs per stream per chunk: warp g
// owns the 32 SPT streams from 32 SPT g on, lane l runs streams 32 SPT g + 32 t + l (t < SPT),
// and each chunk goes out as one 2D tensor store of a CH x 32 SPT box from the warp's tile.
// Rows are CH * 8 bytes, swizzled in 128-byte (CH = 16: piece c of row r at
// r 128 + (c ^ (r & 7)) 16) or 64-byte (CH = 8: r 64 + (c ^ ((r >> 1) & 3)) 16) mode, which
// keeps the lanes' 16-byte stores free of bank conflicts.
// Each step of x2's recurrence needs the previous value, so with one stream per thread the
// issue slots idle while that chain's latency runs out; with two, the compiler interleaves
// two independent chains. Outputs go to the tile two at a time as they are made, so no
// register holds a whole chunk.
template <int FORM, int MAP = 0, int SPT = 1, int CH = kChunk>
__global__ void __launch_bounds__(256) fill_mrg_tma_kernel(const FillParams p, const __grid_constant__ CUtensorMap tmap) {
  static_assert(CH == 16 || CH == 8, "rows of 128 or 64 bytes");
  constexpr uint32_t kRowBytes = CH * 8;
  constexpr uint32_t kWarpTile = 32u * SPT * kRowBytes;
  extern __shared__ uint8_t smem_raw[];
  const uint32_t base = (smem_addr(smem_raw) + 1023u) & ~1023u;
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const uint64_t warp_global = (uint64_t)blockIdx.x * (blockDim.x >> 5) + warp;
  const uint64_t first = warp_global * 32 * SPT;
  if (first >= p.n_streams) return;
  Mrg32k3a g[SPT];
  uint32_t rej[SPT];
  uint32_t rowb[SPT];  // row address with the swizzle's xor pattern or-ed into bits 4..6
  const uint32_t tile = base + (uint32_t)warp * kWarpTile;
#pragma unroll
  for (int t = 0; t < SPT; ++t) {
    const uint64_t stream = first + 32 * t + lane;
    g[t] = stream < p.n_streams ? mrg_load(p.state, stream) : Mrg32k3a{1u, 2u, 3u, 4u, 5u, 6u};
    rej[t] = 0;
    const uint32_t r = 32u * t + (uint32_t)lane;
    rowb[t] = (tile + r * kRowBytes) | ((CH == 16 ? (r & 7u) : ((r >> 1) & 3u)) << 4);
  }
  for (uint64_t x0 = 0; x0 < p.per_stream; x0 += CH) {
    const uint64_t left = p.per_stream - x0;
    if (lane == 0) bulk_wait_read<0>();  // the previous chunk's store has read the tile
    __syncwarp();
    if (left >= (uint64_t)CH) {
#pragma unroll kMrgUnroll
      for (int c = 0; c < CH / 2; ++c) {
        uint64_t v0[SPT], v1[SPT];
        if constexpr (FORM != kFormA) {
#pragma unroll
          for (int t = 0; t < SPT; ++t) mrg_next_pair<FORM, MAP>(g[t], rej[t], p, v0[t], v1[t]);
        } else {
#pragma unroll
          for (int t = 0; t < SPT; ++t) v0[t] = mrg_next_output<FORM, MAP>(g[t], rej[t], p);
#pragma unroll
          for (int t = 0; t < SPT; ++t) v1[t] = mrg_next_output<FORM, MAP>(g[t], rej[t], p);
        }
#pragma unroll
        for (int t = 0; t < SPT; ++t) st_shared_v2(rowb[t] ^ ((uint32_t)c << 4), v0[t], v1[t]);
      }
    } else {
#pragma unroll
      for (int c = 0; c < CH / 2; ++c) {
#pragma unroll
        for (int t = 0; t < SPT; ++t) {
          const uint64_t a = ((uint64_t)(2 * c) < left) ? mrg_next_output<FORM, MAP>(g[t], rej[t], p) : 0ull;
          const uint64_t b = ((uint64_t)(2 * c + 1) < left) ? mrg_next_output<FORM, MAP>(g[t], rej[t], p) : 0ull;
          st_shared_v2(rowb[t] ^ ((uint32_t)c << 4), a, b);
        }
      }
    }
    fence_async_shared();
    __syncwarp();
    if (lane == 0) {  // rows past the last stream and columns past per_stream are clipped
      tma_store_2d(&tmap, tile, (int)x0, (int)first);
      bulk_commit();
    }
  }
  if (lane == 0) bulk_wait_all();
#pragma unroll
  for (int t = 0; t < SPT; ++t) {
    const uint64_t stream = first + 32 * t + lane;
    if (stream < p.n_streams) {
      mrg_store(p.state, stream, g[t]);
      if (p.rejects) p.rejects[stream] = rej[t];
    }
  }
}

// Plain stores (any alignment, host-mapped outputs): each thread writes its own stream.
template <int FORM, int MAP = 0>
__global__ void __launch_bounds__(256) fill_mrg_plain_kernel(const FillParams p) {
  const uint64_t stream = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (stream >= p.n_streams) return;
  Mrg32k3a g = mrg_load(p.state, stream);
  uint32_t rej = 0;
  uint64_t* dst = p.out + stream * p.per_stream;
  for (uint64_t i = 0; i < p.per_stream; ++i) dst[i] = mrg_next_output<FORM, MAP>(g, rej, p);
  mrg_store(p.state, stream, g);
  if (p.rejects) p.rejects[stream] = rej;
}

}  // namespace prngd

namespace prngd_host {

// Division constants of D = (m1 - 1)^2 (normalised by its own shift) and RN(1/D).
static prngd::DivConst mrg_divconst() {
  const uint64_t m = prngd::kMrgM1 - 1u;
  const uint64_t d = m * m;
  prngd::DivConst dc;
  dc.sh = prngd::clz64(d);
  dc.d_norm = d << dc.sh;
  const unsigned __int128 all = ~(unsigned __int128)0;
  dc.v = (uint64_t)(all / dc.d_norm - ((unsigned __int128)1 << 64));
  return dc;
}

namespace {
constexpr int kWarpsPerBlock = 8;
#ifndef PRNGD_MRG_SPT
#define PRNGD_MRG_SPT 1
#endif
#ifndef PRNGD_MRG_CHUNK
#define PRNGD_MRG_CHUNK 16
#endif
constexpr int kSpt = PRNGD_MRG_SPT;    // streams per thread of the TMA path
constexpr int kCh = PRNGD_MRG_CHUNK;   // outputs per stream per staged chunk
constexpr size_t kTmaSmem = (size_t)kWarpsPerBlock * 32 * kSpt * kCh * 8 + 1024;

template <int FORM, int MAP = 0>
cudaError_t launch_mrg_form(const prngd::FillParams& p, const CUtensorMap* map, cudaStream_t s) {
  if (map) {
    const uint64_t per_block = (uint64_t)kWarpsPerBlock * 32 * kSpt;
    const unsigned blocks = (unsigned)((p.n_streams + per_block - 1) / per_block);
    auto k = prngd::fill_mrg_tma_kernel<FORM, MAP, kSpt, kCh>;
    static std::atomic<uint64_t> attr{0};
    const cudaError_t e = prngd::smem_limit_once(k, (int)kTmaSmem, attr);
    if (e != cudaSuccess) return e;
    k<<<blocks, kWarpsPerBlock * 32, kTmaSmem, s>>>(p, *map);
  } else {
    prngd::fill_mrg_plain_kernel<FORM, MAP><<<(unsigned)((p.n_streams + 255) / 256), 256, 0, s>>>(p);
  }
  return cudaGetLastError();
}
}  // namespace

int launch_fill_mrg(prng_ctx* h, uint4* state, uint64_t n_streams, void* out, uint64_t per_stream, int form,
                    uint64_t* rejects, cudaStream_t s, bool allow_tma, int mode) {
  if (n_streams == 0 || per_stream == 0) return PRNG_OK;
  // PRNG_MODE_BALANCED changes no value: it selects form B's FP64 rounding route (form A's MRG
  // conversion is the instruction already)
  if ((mode & ~PRNG_MODE_BALANCED) != 0 ||
      (form != PRNG_FORM_A_FP64 && form != PRNG_FORM_B_INTBITS && form != PRNG_FORM_C_F32PAIR))
    return fail(PRNG_EINVAL, "MRG32k3a streams take forms A, B and C with mode 0");
  if (allow_tma && device_mapped_host(out, nullptr)) allow_tma = false;
  prngd::FillParams p;
  memset(&p, 0, sizeof(p));
  p.state = state;
  p.n_streams = n_streams;
  p.per_stream = per_stream;
  p.out = (uint64_t*)out;
  p.rejects = rejects;
  p.dc = h->dc;
  p.scale = h->scale;
  p.w = 32;
  p.one = 1;
  CUtensorMap map;
  const CUtensorMap* mp =
      (allow_tma && encode_out_map_box(&map, out, n_streams, per_stream, (uint32_t)kCh, 32u * kSpt, 0)) ? &map : nullptr;
  cudaError_t e;
  switch (form) {
    case PRNG_FORM_A_FP64: e = launch_mrg_form<prngd::kFormA>(p, mp, s); break;
    case PRNG_FORM_C_F32PAIR: e = launch_mrg_form<prngd::kFormC>(p, mp, s); break;
    default:
      e = (mode & PRNG_MODE_BALANCED) ? launch_mrg_form<prngd::kFormB, prngd::kMapCvt>(p, mp, s)
                                      : launch_mrg_form<prngd::kFormB>(p, mp, s);
      break;
  }
  if (e != cudaSuccess) return fail(PRNG_ECUDA, "MRG32k3a fill launch: %s", cudaGetErrorString(e));
  return PRNG_OK;
}

}  // namespace prngd_host

using namespace prngd_host;

extern "C" {

int prng_create_mrg32k3a(prng_t* out, uint64_t seed, uint64_t n_streams) {
  if (!out) return fail(PRNG_EINVAL, "out is NULL");
  *out = nullptr;
  if (n_streams == 0 || n_streams > (1ull << 32)) return fail(PRNG_EINVAL, "n_streams must be in [1, 2^32]");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(PRNG_ECUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
  prng_ctx* h = new prng_ctx();
  h->device = dev;
  h->seed = seed;
  h->n_streams = n_streams;
  h->w = 32;
  h->gen = PRNG_GEN_MRG32K3A;
  h->dc = mrg_divconst();
  const uint64_t one = prngd::rn_bits_exact(1, h->dc);  // RN(1/D)
  memcpy(&h->scale, &one, 8);
  e = cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaMalloc(&h->d_state, n_streams * 2 * sizeof(uint4));
  if (e != cudaSuccess) {
    cudaGetLastError();
    delete h;
    return fail(PRNG_ENOMEM, "MRG32k3a state (%llu bytes): %s", (unsigned long long)(n_streams * 32),
                cudaGetErrorString(e));
  }
  prngd::mrg_seed_kernel<<<(unsigned)((n_streams + 255) / 256), 256>>>(h->d_state, n_streams, seed);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(0);
  if (e != cudaSuccess) {
    cudaFree(h->d_state);
    delete h;
    return fail(PRNG_ECUDA, "MRG32k3a seeding: %s", cudaGetErrorString(e));
  }
  *out = h;
  return PRNG_OK;
}

int prng_generator(prng_t h) { return h ? h->gen : -1; }

}  // extern "C"
