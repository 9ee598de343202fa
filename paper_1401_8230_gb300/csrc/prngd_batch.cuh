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

namespace prngd {

struct BatchDesc {       // 64 bytes, built on the host
  uint64_t seed;         // fresh: seed of the streams
  uint64_t first_stream; // fresh: first stream id; resident: first handle stream
  uint64_t length;       // outputs of the request
  uint64_t per_stream;   // row length (even)
  uint64_t* out;         // 16-byte aligned, length outputs
  uint64_t* rejects;     // nullable, one count per row
  uint32_t n_rows;       // streams used
  int32_t form;          // kFormA / kFormB / kFormC
  uint32_t resident;     // 1: rows continue handle streams
  uint32_t pad;
};

struct BatchParams {
  const BatchDesc* desc;          // n_req descriptors (longest rows first)
  const uint64_t* item_prefix;    // n_req + 1 cumulative counts of 32-row items
  const uint32_t* n_req_dev;      // number of requests of this launch (device, so a captured graph can be replayed)
  unsigned long long* ticket;     // item counter, zeroed before each launch
  uint4* state;                   // the handle's resident streams
  DivConst dc;
  double scale;
  int w;
  uint32_t one;
  uint32_t items_per_ticket;
};

constexpr int kSlotPitch = 144;

__device__ __forceinline__ uint64_t ld_shared_u64(uint32_t addr) {
  uint64_t v;
  asm volatile("ld.shared.b64 %0, [%1];" : "=l"(v) : "r"(addr) : "memory");
  return v;
}  // 128-byte row segment + 16 bytes of padding: conflict-free staging

__device__ __forceinline__ void bulk_store_1d(uint64_t* dst, uint32_t src, uint32_t bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(src), "r"(bytes)
               : "memory");
}

// One row (one stream) of `count` outputs into out_row, staged per 16 outputs in this lane's
// shared slot and written with 1D bulk copies (rows start 16-byte aligned: even row length and
// aligned base). An odd final output is written with a plain store.
template <int W, int FORM>
__device__ __forceinline__ void batch_row(XorShift128& st, uint32_t& rej, const FillParams& fp, uint64_t count,
                                          uint64_t* out_row, uint32_t slot) {
  for (uint64_t x0 = 0; x0 < count; x0 += kChunk) {
    uint64_t v[kChunk];
    const uint64_t left = count - x0;
    if (left >= (uint64_t)kChunk) {
      if constexpr ((W == 32 || W == 24) && FORM != kFormA) {
#pragma unroll
        for (int j = 0; j < kChunk; j += 2) next_pair<W, FORM>(st, rej, fp, v[j], v[j + 1]);
      } else {
#pragma unroll
        for (int j = 0; j < kChunk; ++j) v[j] = next_output<W, FORM>(st, rej, fp);
      }
    } else {
#pragma unroll
      for (int j = 0; j < kChunk; ++j) v[j] = (j < (int)left) ? next_output<W, FORM>(st, rej, fp) : 0ull;
    }
    const uint32_t n = left >= (uint64_t)kChunk ? (uint32_t)kChunk : (uint32_t)left;
    const uint32_t even = n & ~1u;
    bulk_wait_read<0>();  // this lane's previous copy has finished reading the slot
#pragma unroll
    for (int c = 0; c < kChunk / 2; ++c) st_shared_v2(slot + 16u * c, v[2 * c], v[2 * c + 1]);
    fence_async_shared();
    if (even) {
      bulk_store_1d(out_row + x0, slot, even * 8u);
      bulk_commit();
    }
    if (n & 1u) out_row[x0 + n - 1] = ld_shared_u64(slot + 8u * (n - 1u));
  }
}

template <int W, int FORM>
__device__ __forceinline__ void batch_item(const BatchDesc& d, uint64_t row, const BatchParams& bp,
                                           const FillParams& fp, uint32_t slot) {
  const bool active = row < d.n_rows;
  uint64_t count = 0;
  if (active) {
    const uint64_t start = row * d.per_stream;
    count = d.length > start ? (d.length - start < d.per_stream ? d.length - start : d.per_stream) : 0;
  }
  if (!active) return;
  XorShift128 st;
  if (d.resident) {
    const uint4 s4 = bp.state[d.first_stream + row];
    st = XorShift128{s4.x, s4.y, s4.z, s4.w};
  } else {
    st = seed_stream(d.seed, d.first_stream + row);
  }
  uint32_t rej = 0;
  if (count) batch_row<W, FORM>(st, rej, fp, count, d.out + row * d.per_stream, slot);
  if (d.resident) bp.state[d.first_stream + row] = make_uint4(st.x, st.y, st.z, st.w);
  if (d.rejects) d.rejects[row] = rej;
}

// Persistent batch kernel: each warp repeatedly takes items_per_ticket items from the
// counter; an item is located by binary search over the per-request item prefix.
template <int W>
__global__ void __launch_bounds__(256) batch_kernel(const BatchParams bp) {
  extern __shared__ uint8_t smem_raw[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t slot = smem_addr(smem_raw) + (uint32_t)(warp * 32 + lane) * kSlotPitch;
  const uint32_t n_req = *bp.n_req_dev;
  const uint64_t total = bp.item_prefix[n_req];
  FillParams fp;
  fp.dc = bp.dc;
  fp.scale = bp.scale;
  fp.w = bp.w;
  fp.one = bp.one;
  for (;;) {
    unsigned long long first = 0;
    if (lane == 0) first = atomicAdd(bp.ticket, (unsigned long long)bp.items_per_ticket);
    first = __shfl_sync(0xffffffffu, first, 0);
    if (first >= total) break;
    const uint64_t last = first + bp.items_per_ticket < total ? first + bp.items_per_ticket : total;
    for (uint64_t item = first; item < last; ++item) {
      uint32_t lo = 0, hi = n_req;  // largest r with prefix[r] <= item
      while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (bp.item_prefix[mid] <= item) lo = mid; else hi = mid;
      }
      const BatchDesc d = bp.desc[lo];
      const uint64_t row = (item - bp.item_prefix[lo]) * 32 + lane;
      switch (d.form) {
        case kFormA: batch_item<W, kFormA>(d, row, bp, fp, slot); break;
        case kFormC: batch_item<W, kFormC>(d, row, bp, fp, slot); break;
        default: batch_item<W, kFormB>(d, row, bp, fp, slot); break;
      }
    }
  }
  bulk_wait_all();
}

}  // namespace prngd
