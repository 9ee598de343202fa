// prngd_internal.h -- the handle behind prng_t and helpers shared by the library's
// translation units. Not part of the public ABI.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "prngd.h"
#include "prngd_math.cuh"

namespace prngd {
struct FillParams;
struct BatchParams;
}

namespace prngd_host {
struct BatchEngine;
struct BatchShape {
  int warps_per_block;
  int blocks_per_sm;
  int items_per_ticket;
  int outputs_per_chunk;  // outputs a lane makes between the warp's tensor stores (16 or 32)
};
}  // namespace prngd_host

struct prng_ctx {
  int gen = PRNG_GEN_XORSHIFT128;  // base generator of the streams
  int device;
  uint64_t seed;
  uint64_t n_streams;
  int w;
  uint4* d_state;       // the streams' states, resident between calls: one uint4 per xorshift128
                        // stream, two per MRG32k3a stream
  prngd::DivConst dc;   // exact-division constants of D = (2^w - 1)^2
  double scale;         // C_w = RN(1/D)
  int num_sms;          // multiprocessors of the handle's device
  // staging for prng_fill_f64_host (allocated on first use)
  void* d_stage[2] = {nullptr, nullptr};
  size_t stage_bytes = 0;
  uint64_t* d_rej_stage = nullptr;
  cudaStream_t io_stream[2] = {nullptr, nullptr};
  // batched requests (created on first use)
  prngd_host::BatchEngine* batch = nullptr;
  // split-fill scratch (grown on demand)
  void* split_mem = nullptr;
  size_t split_bytes = 0;
  uint64_t split_table_seg = 0;     // segment length the jump table in the scratch was built for
  void* split_table_mem = nullptr;  // where that table lives
  int split_table_digits = 0;       // digits of the segment index it covers
};

namespace prngd_host {
int fail(int code, const char* fmt, ...);
int check_handle_device(prng_ctx* h);
// Output arguments of a fill: a device rejects array (nullable) of 8-byte aligned words, and at
// most 2^60 outputs in all (n_streams * per_stream), so that every byte offset fits in 64 bits.
int check_fill_extent(prng_ctx* h, uint64_t per_stream, const void* d_rejects);
constexpr uint64_t kMaxOutputs = 1ull << 60;
int launch_fill(prng_ctx* h, uint4* state, uint64_t n_streams, void* out, uint64_t per_stream, int form,
                uint64_t* rejects, cudaStream_t s, bool allow_tma, int mode = 0);
// Every PRNG_MODE_* bit an entry point accepts.
constexpr int kAllModes = PRNG_MODE_EQ5 | PRNG_MODE_ONE_MINUS | PRNG_MODE_SINGLE_REDRAW | PRNG_MODE_BALANCED;
// The kernels' MAP bits of a mode: the map bits (mode & 3), and for forms A and B the balanced
// route of PRNG_MODE_BALANCED (kMapCvt = 4 in prngd_fill.cuh).
inline int map_bits_of(int form, int mode) {
  return (mode & (PRNG_MODE_EQ5 | PRNG_MODE_ONE_MINUS)) |
         (((form == PRNG_FORM_B_INTBITS || form == PRNG_FORM_A_FP64) && (mode & PRNG_MODE_BALANCED)) ? 4 : 0);
}
// Kernels for the Eq. 5 / 1 - z maps, the balanced routes and form L (prngd_modes.cu,
// prngd_modes_fast.cu): `map` as map_bits_of; `tmap` is null for the plain store path.
cudaError_t launch_fill_map(const prngd::FillParams& p, int form, int map, const CUtensorMap* tmap, cudaStream_t s);
cudaError_t launch_fill_map_fast(const prngd::FillParams& p, int form, int map, const CUtensorMap* tmap,
                                 cudaStream_t s, bool shift = false);
int host_fill(prng_ctx* h, double* host_out, uint64_t per_stream, int form, uint64_t* host_rejects);
bool device_mapped_host(const void* p, void** dev);
bool encode_out_map(CUtensorMap* map, void* out, uint64_t n_streams, uint64_t per_stream);
bool encode_out_map_box(CUtensorMap* map, void* out, uint64_t n_streams, uint64_t per_stream, uint32_t box_x,
                        uint32_t box_y, uint64_t pitch);
void release_aux(prng_ctx* h);
void release_split(prng_ctx* h);
int launch_fill_mrg(prng_ctx* h, uint4* state, uint64_t n_streams, void* out, uint64_t per_stream, int form,
                    uint64_t* rejects, cudaStream_t s, bool allow_tma, int mode);
// State of stream s within the handle's state array (uint4 units per stream depend on the generator).
inline uint4* state_at(prng_ctx* h, uint64_t s) { return h->d_state + (h->gen == PRNG_GEN_MRG32K3A ? 2 * s : s); }
// PRNG_EINVAL unless the handle's streams are xorshift128 (paths built on its GF(2) structure,
// its fast conversions or its 16-byte state).
int require_xorshift(prng_ctx* h, const char* what);
// Division constants of D = (2^w - 1)^2 and the form-A scale RN(1/D).
prngd::DivConst make_divconst(int w);
double scale_constant(const prngd::DivConst& dc);
// Mode-dependent constants of FillParams (reject rule, Eq. 5 division constants, form L).
void set_mode_constants(prngd::FillParams& p, int w, int mode);
void release_batch(prng_ctx* h);
BatchShape default_batch_shape(int num_sms);
// The batch kernel for requests of any form and mode at w = W (32, 24, or 0 for the generic
// code); one translation unit defines each.
// `blocks` blocks of the shape's warps, shared memory for the item prefix of max_req requests.
template <int W>
cudaError_t launch_batch_any_mode_w(const prngd::BatchParams& p, const BatchShape& sh, unsigned blocks, int max_req,
                                    cudaStream_t s);
template <>
cudaError_t launch_batch_any_mode_w<32>(const prngd::BatchParams&, const BatchShape&, unsigned, int, cudaStream_t);
template <>
cudaError_t launch_batch_any_mode_w<24>(const prngd::BatchParams&, const BatchShape&, unsigned, int, cudaStream_t);
template <>
cudaError_t launch_batch_any_mode_w<0>(const prngd::BatchParams&, const BatchShape&, unsigned, int, cudaStream_t);
// prng_submit with an optional cap on the items each warp takes (items_per_warp > 0): the batch
// is then launched directly (no graph) with just enough blocks to cover its items under the
// cap, so that its blocks finish, and free their SM slots, every few items instead of at the
// end of the batch. The serving loop uses it; 0 is prng_submit.
// warps (> 0) overrides the shape's warps per block for a capped launch.
int submit_capped(prng_ctx* h, const prng_request* reqs, int n, uint64_t* ticket, cudaStream_t s,
                  uint32_t items_per_warp, int warps = 0);
int set_batch_shape(prng_ctx* h, const BatchShape& sh);
int get_batch_shape(prng_ctx* h, BatchShape* sh);
}  // namespace prngd_host
