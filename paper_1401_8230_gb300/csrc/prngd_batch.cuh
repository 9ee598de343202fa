// prngd_batch.cuh -- many fill requests of uneven length in one persistent launch.
//
// A request is a stream-major block of rows: row j holds the outputs of one stream, in order.
// Fresh requests use streams first_stream + j of their own seed (rows of `chunk` outputs, the
// last one shorter); resident requests continue a range of the handle's device-resident
// streams (row j = handle stream first_stream + j, rows of per_stream outputs, the tail rows
// shorter or empty). A work item is 32 consecutive rows of one request; warps take items from
// a device counter, so one warp always works on one request (its form is warp-uniform). The
// result never depends on the launch shape or on which warp takes which item.
#pragma once
#include <stdint.h>

#include "prngd_fill.cuh"
#include "prngd_launch.h"

namespace prngd {

constexpr uint32_t kModeSingle = 4;      // BatchDesc::mode bit: Algorithm 1's single-redraw rejects
constexpr uint32_t kModeBalanced = 8;    // BatchDesc::mode bit: PRNG_MODE_BALANCED (forms A and B)

struct BatchDesc {       // 64 bytes, built on the host
  uint64_t seed;         // fresh: seed of the streams
  uint64_t first_stream; // fresh: first stream id; resident: first handle stream
  uint64_t length;       // outputs of the request
  uint64_t per_stream;   // row length (even)
  uint64_t* out;         // 16-byte aligned, length outputs
  uint64_t* rejects;     // nullable, one count per row
  uint32_t n_rows;       // streams used
  int32_t form;          // kFormA / kFormB / kFormC / kFormL
  uint8_t resident;      // 1: rows continue handle streams
  uint8_t shift;         // 1: rows start 16 bytes into a 32-byte sector; the request's map then
                         // starts 2 outputs into each row (see batch_item_full)
  uint16_t mode;         // PRNG_MODE_* bits: Eq. 5 map, 1 - z, Algorithm 1's single redraw
  uint32_t full_rows;    // rows 0 .. full_rows-1 hold per_stream outputs and are covered by the
                         // request's tensor map (0: no map, plain stores only)
};

struct BatchParams {
  const BatchDesc* desc;          // n_req descriptors (longest rows first)
  const CUtensorMap* maps;        // one per descriptor: 2D map of its full rows (used when full_rows > 0)
  const uint32_t* meta;           // meta[0] = n_req, meta[1 .. n_req + 1] = cumulative counts of
                                  // 32-row items (< 2^32); device memory, so a captured graph replays
  unsigned long long* ticket;     // item counter, zeroed before each launch
  uint4* state;                   // the handle's resident streams
  DivConst dc;
  double scale;
  int w;
  uint32_t one;
  uint32_t items_per_ticket;
  uint32_t items_per_warp;        // 0: a warp takes items until none is left; else it stops
                                  // after taking at least this many (the grid covers the batch)
  DivConst ec;                    // Eq. 5: constants of D - 2
  double scale5;                  // Eq. 5, form A: RN((1 - k^2)/(D - 2))
  double k;                       // form L: 2^-w and its folded constants under Eq. 4 and Eq. 6
  double l1_eq4, l2_eq4, l1_eq5, l2_eq5;
};

constexpr int kSlotPitch = 144;

  // 128-byte row segment + 16 bytes of padding: conflict-free staging


__device__ __forceinline__ void tma_store_2d_global_map(const CUtensorMap* map, uint32_t src, int x, int y) {
  asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%2, %3}], [%1];" ::"l"(map), "r"(src), "r"(x),
               "r"(y)
               : "memory");
}

__device__ __forceinline__ uint4 ld_shared_v4(uint32_t addr) {
  uint4 v;
  asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];" : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "r"(addr) : "memory");
  return v;
}

// Generates the next kChunk outputs of the lane's row (all of them exist) and stages them as
// row `lane` of the warp's tile (128-byte swizzle: piece c of row r at r*128 + ((c ^ (r & 7)) *
// 16)). Four outputs per iteration of a loop that is not unrolled: with warps that drift apart
// in a persistent launch, a fully unrolled chunk (eight pairs, each with its inline medium path)
// no longer fits the instruction cache. Lane 0 waits for the warp's previous tensor store to
// have read the tile before the first piece is written.
// CVT: the outputs of each 4-output step rounded by the conversion instruction (cvt_group_mask).
// CH = 32: 32 outputs as two 32 x 16 sub-tiles 4 KiB apart (pieces 8..15 of the row in the
// second), each with the same swizzle.
template <int W, int FORM, int MAP, uint32_t CVT, int CH = kChunk>
__device__ __forceinline__ void stage_full_chunk(XorShift128& st, uint32_t& rej, const FillParams& fp,
                                                 uint32_t my_row, uint32_t sw, int lane) {
  static_assert(CH == kChunk || CH == 2 * kChunk, "one or two sub-tiles");
  // my_row has zero bits 4..6 (1024-byte aligned tile, 128-byte rows): piece c lies at
  // (my_row | (sw << 4)) ^ 16c, and the loop counts c4 = 16c
  const uint32_t rowb = my_row | (sw << 4);
#pragma unroll 1
  for (uint32_t c4 = 0; c4 < (uint32_t)CH * 8u; c4 += 32u) {
    uint64_t a0, a1, b0, b1;
    if constexpr ((W == 32 || W == 24) && (FORM == kFormB || FORM == kFormC)) {
      next_pair<W, FORM, MAP>(st, rej, fp, a0, a1, CVT & 1u, (CVT >> 1) & 1u);
      next_pair<W, FORM, MAP>(st, rej, fp, b0, b1, (CVT >> 2) & 1u, (CVT >> 3) & 1u);
    } else {
      a0 = next_output<W, FORM, MAP>(st, rej, fp);
      a1 = next_output<W, FORM, MAP>(st, rej, fp);
      b0 = next_output<W, FORM, MAP>(st, rej, fp);
      b1 = next_output<W, FORM, MAP>(st, rej, fp);
    }
    if (c4 == 0) {  // warp-uniform
      if (lane == 0) bulk_wait_read<0>();
      __syncwarp();
    }
    uint32_t a = rowb ^ c4;
    if constexpr (CH == 2 * kChunk) a = (rowb + ((c4 >> 7) << 12)) ^ (c4 & 0x70u);  // sub-tile c / 8
    st_shared_v2(a, a0, a1);
    st_shared_v2(a ^ 16u, b0, b1);
  }
}

// The conversion constants of a batch launch, as the fill code takes them.
template <int MAP = 0>
__device__ __forceinline__ FillParams fill_params_of(const BatchParams& bp, uint32_t single = 0) {
  FillParams fp;
  fp.dc = bp.dc;
  fp.scale = bp.scale;
  fp.w = bp.w;
  fp.one = bp.one;
  fp.single = single;
  fp.ec = bp.ec;
  fp.scale5 = bp.scale5;
  fp.k = bp.k;
  fp.l1 = (MAP & kMapEq5) ? bp.l1_eq5 : bp.l1_eq4;
  fp.l2 = (MAP & kMapEq5) ? bp.l2_eq5 : bp.l2_eq4;
  return fp;
}

struct RowState {  // a row's stream and reject count, passed by value to out-of-line code
  XorShift128 st;
  uint32_t rej;
};

// Generates the lane's next min(left, kChunk) outputs (zeros after them) and stages them as
// above; the whole chunk is written, after the same wait. Out of line: it runs once per row at
// most, at the row's end. `bp` is the launch's grid constant.
template <int W, int FORM, int MAP>
__device__ __noinline__ RowState stage_partial_chunk(RowState rs, const BatchParams& bp, uint32_t single,
                                                     uint32_t my_row, uint32_t sw, int lane, uint32_t left) {
  const FillParams fp = fill_params_of<MAP>(bp, single);
  XorShift128 st = rs.st;
  uint32_t rej = rs.rej;
  uint64_t v[kChunk];
#pragma unroll
  for (int j = 0; j < kChunk; ++j) v[j] = ((uint32_t)j < left) ? next_output<W, FORM, MAP>(st, rej, fp) : 0ull;
  if (lane == 0) bulk_wait_read<0>();
  __syncwarp();
#pragma unroll
  for (int c = 0; c < kChunk / 2; ++c) st_shared_v2(my_row + (((uint32_t)c ^ sw) << 4), v[2 * c], v[2 * c + 1]);
  return RowState{st, rej};
}

// The first two outputs of a row whose request is shifted (BatchDesc::shift). Out of line: once
// per row.
struct RowHead {
  RowState rs;
  uint64_t v0, v1;
};
template <int W, int FORM, int MAP>
__device__ __noinline__ RowHead row_head(RowState rs, const BatchParams& bp, uint32_t single) {
  const FillParams fp = fill_params_of<MAP>(bp, single);
  const uint64_t v0 = next_output<W, FORM, MAP>(rs.st, rs.rej, fp);
  const uint64_t v1 = next_output<W, FORM, MAP>(rs.st, rs.rej, fp);
  return RowHead{rs, v0, v1};
}

// Stream state of row `row` of a request at its first output.
__device__ __forceinline__ XorShift128 item_row_state(const BatchDesc* __restrict__ dp, const BatchParams& bp,
                                                      uint64_t row) {
  if (dp->resident) {
    const uint4 s4 = bp.state[dp->first_stream + row];
    return XorShift128{s4.x, s4.y, s4.z, s4.w};
  }
  return seed_stream(dp->seed, dp->first_stream + row);
}

// An item of 32 full rows (every row holds per_stream outputs): rows row0 .. row0 + 31 of a
// request, one per lane. Per chunk of 16 outputs the warp stages its 32 x 16 tile and lane 0
// writes it with one 2D tensor store through the request's map (columns past per_stream are
// clipped). With CH = 32 each lane makes 32 outputs per chunk while 32 remain, written as two
// stores of the two sub-tiles, and the rest of the row in chunks of 16. fp carries the
// request's reject rule.
// A shifted request (rows starting 16 bytes into a 32-byte sector) would have every store begin
// and end in half a sector. Its map instead starts 2 outputs into each row (16 bytes further,
// on a sector boundary, with the rows' own pitch) and covers outputs 2 .. per_stream - 1: each
// lane keeps its row's first two outputs in registers and writes them as one 16-byte store
// after the row, when the lane below writes the other half of that sector (its row's last two
// outputs).
template <int W, int FORM, int MAP, uint32_t CVT, int CH = kChunk>
__device__ __forceinline__ void batch_item_full(const BatchDesc* __restrict__ dp, const CUtensorMap* map,
                                                uint64_t row0, const BatchParams& bp, const FillParams& fp,
                                                uint32_t tile, int lane) {
  const uint64_t row = row0 + lane;
  XorShift128 st = item_row_state(dp, bp, row);
  uint32_t rej = 0;
  const uint32_t my_row = tile + (uint32_t)lane * 128u;
  const uint32_t sw = (uint32_t)(lane & 7);
  if (lane == 0)  // the map was rewritten by a host copy since an earlier batch may have used this slot
    asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(map) : "memory");
  const bool shift = dp->shift != 0;  // warp-uniform
  uint64_t head0 = 0, head1 = 0;
  if (shift) {
    const RowHead rh = row_head<W, FORM, MAP>(RowState{st, rej}, bp, fp.single);
    st = rh.rs.st;
    rej = rh.rs.rej;
    head0 = rh.v0;
    head1 = rh.v1;
  }
  const uint32_t per = (uint32_t)dp->per_stream - (shift ? 2u : 0u);  // outputs the map covers
  uint32_t x0 = 0;
  if constexpr (CH == 2 * kChunk) {
#pragma unroll 1
    for (; per - x0 >= (uint32_t)CH; x0 += CH) {
      stage_full_chunk<W, FORM, MAP, CVT, CH>(st, rej, fp, my_row, sw, lane);
      fence_async_shared();
      __syncwarp();
      if (lane == 0) {
        tma_store_2d_global_map(map, tile, (int)x0, (int)row0);
        tma_store_2d_global_map(map, tile + (uint32_t)kTileBytes, (int)(x0 + kChunk), (int)row0);
        bulk_commit();
      }
    }
  }
#pragma unroll 1
  for (; x0 < per; x0 += kChunk) {
    const uint32_t left = per - x0;
    if (left >= (uint32_t)kChunk) {
      stage_full_chunk<W, FORM, MAP, CVT>(st, rej, fp, my_row, sw, lane);
    } else {
      const RowState rs = stage_partial_chunk<W, FORM, MAP>(RowState{st, rej}, bp, fp.single, my_row, sw, lane, left);
      st = rs.st;
      rej = rs.rej;
    }
    fence_async_shared();
    __syncwarp();
    if (lane == 0) {
      tma_store_2d_global_map(map, tile, (int)x0, (int)row0);
      bulk_commit();
    }
  }
  if (shift) {
    ulonglong2* head = (ulonglong2*)(dp->out + row * dp->per_stream);  // 16-byte aligned
    *head = make_ulonglong2(head0, head1);
  }
  if (dp->resident) bp.state[dp->first_stream + row] = make_uint4(st.x, st.y, st.z, st.w);
  uint64_t* rejects = dp->rejects;
  if (rejects) rejects[row] = rej;
}

// Any other item (a request's last rows: ragged, shorter, or past n_rows), kept out of line so
// the hot loop above stays small. The warp stages the tile as above and stores it row by row:
// lane (r, q) stores piece q of row k*4 + r, so each store instruction covers four 128-byte row
// segments; rows are 16-byte aligned and a row's odd last output is stored as 8 bytes.
template <int W, int FORM, int MAP>
__device__ __noinline__ void batch_item_ragged(const BatchDesc* __restrict__ dp, uint64_t row0, const BatchParams& bp,
                                               uint32_t tile, int lane) {
  const uint32_t single = (dp->mode & kModeSingle) ? 1u : 0u;
  const FillParams fp = fill_params_of<MAP>(bp, single);
  const uint64_t row = row0 + lane;
  const uint32_t n_rows = dp->n_rows;
  uint32_t count = 0;  // outputs of this lane's row (row length < 2^32, checked on the host)
  XorShift128 st{1u, 2u, 3u, 4u};
  if (row < n_rows) {
    const uint64_t per = dp->per_stream, length = dp->length, start = row * per;
    if (length > start) count = (uint32_t)(length - start < per ? length - start : per);
    st = item_row_state(dp, bp, row);
  }
  uint32_t rej = 0;
  const uint32_t my_row = tile + (uint32_t)lane * 128u;
  const uint32_t sw = (uint32_t)(lane & 7);
  const uint32_t c0 = __shfl_sync(0xffffffffu, count, 0);
  const bool uniform = __all_sync(0xffffffffu, count == c0);
  const uint32_t max_count = __reduce_max_sync(0xffffffffu, count);
  const uint32_t q = (uint32_t)(lane & 7);
#pragma unroll 1
  for (uint32_t x0 = 0; x0 < max_count; x0 += kChunk) {
    const uint32_t left = count > x0 ? count - x0 : 0u;
    if (__all_sync(0xffffffffu, left >= (uint32_t)kChunk)) {
      stage_full_chunk<W, FORM, MAP, cvt_group_mask<FORM, W, MAP>()>(st, rej, fp, my_row, sw, lane);
    } else {
      const RowState rs = stage_partial_chunk<W, FORM, MAP>(RowState{st, rej}, bp, single, my_row, sw, lane, left);
      st = rs.st;
      rej = rs.rej;
    }
    __syncwarp();
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const uint32_t r = (uint32_t)(k * 4) + ((uint32_t)lane >> 3);
      const uint32_t cr = uniform ? c0 : __shfl_sync(0xffffffffu, count, (int)r);  // warp-uniform branch
      const uint32_t rl = cr > x0 ? cr - x0 : 0u;  // outputs of row r in this chunk
      if (2u * q < rl) {
        uint64_t* dst = dp->out + (row0 + r) * dp->per_stream + x0 + 2u * q;
        const uint4 val = ld_shared_v4(tile + r * 128u + ((q ^ (r & 7u)) << 4));
        if (2u * q + 1u < rl) {
          *(uint4*)dst = val;
        } else {
          *dst = ((uint64_t)val.y << 32) | val.x;
        }
      }
    }
  }
  if (row < n_rows) {
    if (dp->resident) bp.state[dp->first_stream + row] = make_uint4(st.x, st.y, st.z, st.w);
    uint64_t* rejects = dp->rejects;
    if (rejects) rejects[row] = rej;
  }
}

// fp: the launch's constants for MAP with the request's reject rule; CVT as for stage_full_chunk.
template <int W, int FORM, int MAP = 0, uint32_t CVT = cvt_group_mask<FORM, W, MAP>(), int CH = kChunk>
__device__ __forceinline__ void batch_item(const BatchDesc* __restrict__ dp, const CUtensorMap* map, uint64_t row0,
                                           const BatchParams& bp, const FillParams& fp, uint32_t tile, int lane) {
  if (row0 + 32 <= dp->full_rows)  // warp-uniform
    batch_item_full<W, FORM, MAP, CVT, CH>(dp, map, row0, bp, fp, tile, lane);
  else
    batch_item_ragged<W, FORM, MAP>(dp, row0, bp, tile, lane);
}

// An item of a request with any form and map, out of line (one function per pair). Forms B
// and C keep the w-specific fast paths at w = 32 and 24; forms A and L take the generic code,
// as their fills do.
template <int W, int FORM, int MAP>
__device__ __noinline__ void batch_item_fm(const BatchDesc* __restrict__ dp, const CUtensorMap* map, uint64_t row0,
                                           const BatchParams& bp, uint32_t tile, int lane) {
  const FillParams fp = fill_params_of<MAP>(bp, (dp->mode & kModeSingle) ? 1u : 0u);
  constexpr int WI = ((W == 32 || W == 24) && (FORM == kFormB || FORM == kFormC)) ? W : 0;
  batch_item<WI, FORM, MAP>(dp, map, row0, bp, fp, tile, lane);
}

template <int W, int FORM>
__device__ __forceinline__ void batch_item_form_any_map(const BatchDesc* __restrict__ dp, const CUtensorMap* map,
                                                        uint64_t row0, const BatchParams& bp, uint32_t tile, int lane) {
  if constexpr (FORM == kFormB || FORM == kFormA) {  // the balanced routes
    if (dp->mode & kModeBalanced) {
      switch (dp->mode & (kMapEq5 | kMapOneMinus)) {
        case 0: batch_item_fm<W, FORM, kMapCvt>(dp, map, row0, bp, tile, lane); break;
        case kMapEq5: batch_item_fm<W, FORM, kMapCvt | kMapEq5>(dp, map, row0, bp, tile, lane); break;
        case kMapOneMinus: batch_item_fm<W, FORM, kMapCvt | kMapOneMinus>(dp, map, row0, bp, tile, lane); break;
        default: batch_item_fm<W, FORM, kMapCvt | kMapEq5 | kMapOneMinus>(dp, map, row0, bp, tile, lane); break;
      }
      return;
    }
  }
  switch (dp->mode & (kMapEq5 | kMapOneMinus)) {
    case 0: batch_item_fm<W, FORM, 0>(dp, map, row0, bp, tile, lane); break;
    case kMapEq5: batch_item_fm<W, FORM, kMapEq5>(dp, map, row0, bp, tile, lane); break;
    case kMapOneMinus: batch_item_fm<W, FORM, kMapOneMinus>(dp, map, row0, bp, tile, lane); break;
    default: batch_item_fm<W, FORM, kMapEq5 | kMapOneMinus>(dp, map, row0, bp, tile, lane); break;
  }
}

// Persistent batch kernel: each warp repeatedly takes items_per_ticket items from the
// counter. The per-request item prefix is copied into shared memory once per block; an item
// is located by binary search there, or directly when it falls in the warp's last request.
// FORM_ALL >= 0: every request has form FORM_ALL and mode 0 (Eq. 4, pair rejects), which keeps
// the code and its register footprint to one form; -1: forms A, B and C with mode 0 (per-item
// switch, inlined; form A converts on the FP64 pipe, see kFormAF); kAnyMode: any form and mode (per-item call of an out-of-line function).
// In the first two the reject rule is fixed at compile time, so the hot loop carries the code
// of one rule only.
constexpr int kAnyMode = -2;
// kFormBBalanced: every request is form B with exactly PRNG_MODE_BALANCED (form B's values with
// 3 of 4 outputs rounded on the FP64 pipe), in a single-form kernel like FORM_ALL = kFormB.
constexpr int kFormBBalanced = 3;

// The mixed-form kernel gives its FP64 pipe to form A's conversion and rounds forms B and C with
// integer operations. Measured on the batch of forms A/B/C interleaved (Gsamples/s): this 630;
// A, B 1 in 2, C 1 in 2 on the FP64 pipe 560; A, B 3 in 4, C all 468; A by integers, B 3 in 4,
// C all 511.
constexpr int kMixA = kFormAF;
constexpr uint32_t kMixCvtB = 0u, kMixCvtC = 0u;

// CH: outputs per lane per staged chunk of full items (kChunk, or 2 kChunk in two sub-tiles);
// the any-mode kernel and ragged items stage kChunk at a time.
template <int W, int FORM_ALL, int CH = kChunk>
__global__ void __launch_bounds__(256, 3) batch_kernel(const __grid_constant__ BatchParams bp) {
  constexpr uint32_t kWarpTile = (uint32_t)CH * 32u * 8u;
  extern __shared__ uint8_t smem_raw[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int warps = blockDim.x >> 5;
  const uint32_t n_req = bp.meta[0];
  const uint32_t pad = (1024u - (smem_addr(smem_raw) & 1023u)) & 1023u;  // tiles 1024-byte aligned (swizzle)
  const uint32_t tile = smem_addr(smem_raw) + pad + (uint32_t)warp * kWarpTile;
  uint32_t* prefix = (uint32_t*)(smem_raw + pad + (size_t)warps * kWarpTile);
  for (uint32_t i = threadIdx.x; i <= n_req; i += blockDim.x) prefix[i] = bp.meta[1 + i];
  __syncthreads();
  const uint32_t total = prefix[n_req];
  const FillParams fp = fill_params_of(bp);
  uint32_t r = 0;
  uint32_t taken = 0;
  for (;;) {
    if (bp.items_per_warp && taken >= bp.items_per_warp) break;  // warp-uniform
    unsigned long long first = 0;
    if (lane == 0) first = atomicAdd(bp.ticket, (unsigned long long)bp.items_per_ticket);
    first = __shfl_sync(0xffffffffu, first, 0);
    if (first >= total) break;
    const uint32_t last = (uint32_t)(first + bp.items_per_ticket < total ? first + bp.items_per_ticket : total);
    taken += last - (uint32_t)first;
#pragma unroll 1
    for (uint32_t item = (uint32_t)first; item < last; ++item) {
      if (item < prefix[r] || item >= prefix[r + 1]) {  // largest r with prefix[r] <= item
        uint32_t lo = 0, hi = n_req;
        while (hi - lo > 1) {
          const uint32_t mid = (lo + hi) >> 1;
          if (prefix[mid] <= item) lo = mid; else hi = mid;
        }
        r = lo;
      }
      const BatchDesc* dp = bp.desc + r;
      const uint64_t row0 = (uint64_t)(item - prefix[r]) * 32;
      if constexpr (FORM_ALL == kAnyMode) {
        switch (dp->form) {
          case kFormA: batch_item_form_any_map<W, kFormA>(dp, bp.maps + r, row0, bp, tile, lane); break;
          case kFormC: batch_item_form_any_map<W, kFormC>(dp, bp.maps + r, row0, bp, tile, lane); break;
          case kFormL: batch_item_form_any_map<W, kFormL>(dp, bp.maps + r, row0, bp, tile, lane); break;
          default: batch_item_form_any_map<W, kFormB>(dp, bp.maps + r, row0, bp, tile, lane); break;
        }
      } else if constexpr (FORM_ALL == kFormBBalanced) {
        batch_item<W, kFormB, kMapCvt, cvt_group_mask<kFormB, W, kMapCvt>(), CH>(dp, bp.maps + r, row0, bp, fp, tile,
                                                                                lane);
      } else if constexpr (FORM_ALL >= 0) {
        batch_item<W, FORM_ALL, 0, cvt_group_mask<FORM_ALL, W, 0>(), CH>(dp, bp.maps + r, row0, bp, fp, tile, lane);
      } else {
        switch (dp->form) {
          case kFormA:
            batch_item<W, kMixA, 0, cvt_group_mask<kMixA, W, 0>(), CH>(dp, bp.maps + r, row0, bp, fp, tile, lane);
            break;
          case kFormC: batch_item<W, kFormC, 0, kMixCvtC, CH>(dp, bp.maps + r, row0, bp, fp, tile, lane); break;
          default: batch_item<W, kFormB, 0, kMixCvtB, CH>(dp, bp.maps + r, row0, bp, fp, tile, lane); break;
        }
      }
    }
  }
  if (lane == 0) bulk_wait_all();
}

// Host: one launch of batch_kernel<W, FORM_ALL, CH>, `blocks` blocks of `warps` warps; the
// dynamic shared memory holds the warps' tiles and the item prefix of up to max_req requests.
template <int W, int FORM_ALL, int CH = kChunk>
cudaError_t launch_batch_kernel(const BatchParams& p, int warps, unsigned blocks, int max_req, cudaStream_t s) {
  auto k = batch_kernel<W, FORM_ALL, CH>;
  const size_t tile = (size_t)CH * 32 * 8;
  const size_t smem = 1024 + (size_t)warps * tile + 4 * ((size_t)max_req + 1);
  static std::atomic<uint64_t> attr{0};  // the largest launch: 8 warps, 4096 requests
  const cudaError_t e = prngd::smem_limit_once(k, (int)(1024 + 8 * tile + 4 * (4096 + 1)), attr);
  if (e != cudaSuccess) return e;
  k<<<blocks, warps * 32, smem, s>>>(p);
  return cudaGetLastError();
}

}  // namespace prngd
