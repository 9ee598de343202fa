// prngd_convert.cu -- the method's conversion applied to given base draws (prng_convert_pairs):
// each accepted pair (u1, u2) goes through the same device code as the fills (PTX fast paths,
// medium paths, exact division; Eq. 4 or Eq. 5, 1 - z; forms A, B, C and L). At w = 32 under
// Eq. 4, pair i is rounded by the route the fills use for output i of a row (integer
// normalisation or the conversion instruction), so inputs placed at positions 0 .. 3 reach both.
#include <cuda.h>
#include <cuda_runtime.h>
#include <string.h>

#include "prngd_fill.cuh"
#include "prngd_internal.h"

namespace prngd {

template <int W, int FORM, int MAP>
__global__ void convert_pairs_kernel(const FillParams p, const uint32_t* __restrict__ u1s,
                                     const uint32_t* __restrict__ u2s, uint64_t n, uint64_t* __restrict__ out) {
  const uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint32_t top = (p.w == 32) ? 0xFFFFFFFFu : ((1u << p.w) - 1u);
  const uint32_t u1 = u1s[i] & top, u2 = u2s[i] & top;
  // pair i takes the rounding route the fills give output i of a row (cvt_group_mask)
  const bool cvt = ((cvt_group_mask<FORM, W, MAP>() >> (i & 3)) & 1u) != 0;
  out[i] = accepted(u1, top) ? convert_accepted<W, FORM, MAP>(u1, u2, p, cvt) : ~0ull;
}

}  // namespace prngd

namespace prngd_host {
namespace {

template <int W, int FORM, int MAP>
cudaError_t launch_convert(const prngd::FillParams& p, const uint32_t* u1, const uint32_t* u2, uint64_t n,
                           uint64_t* out, cudaStream_t s) {
  prngd::convert_pairs_kernel<W, FORM, MAP><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(p, u1, u2, n, out);
  return cudaGetLastError();
}

template <int W, int FORM>
cudaError_t by_map(int map, const prngd::FillParams& p, const uint32_t* u1, const uint32_t* u2, uint64_t n,
                   uint64_t* out, cudaStream_t s) {
  constexpr int E = prngd::kMapEq5, O = prngd::kMapOneMinus, V = prngd::kMapCvt;
  if constexpr (FORM == prngd::kFormB || FORM == prngd::kFormA) {  // the balanced routes
    switch (map) {
      case V: return launch_convert<W, FORM, V>(p, u1, u2, n, out, s);
      case V | E: return launch_convert<W, FORM, V | E>(p, u1, u2, n, out, s);
      case V | O: return launch_convert<W, FORM, V | O>(p, u1, u2, n, out, s);
      case V | E | O: return launch_convert<W, FORM, V | E | O>(p, u1, u2, n, out, s);
      default: break;
    }
  }
  switch (map & (E | O)) {
    case 0: return launch_convert<W, FORM, 0>(p, u1, u2, n, out, s);
    case E: return launch_convert<W, FORM, E>(p, u1, u2, n, out, s);
    case O: return launch_convert<W, FORM, O>(p, u1, u2, n, out, s);
    default: return launch_convert<W, FORM, E | O>(p, u1, u2, n, out, s);
  }
}

template <int W>
cudaError_t by_form(int form, int map, const prngd::FillParams& p, const uint32_t* u1, const uint32_t* u2, uint64_t n,
                    uint64_t* out, cudaStream_t s) {
  switch (form) {
    case PRNG_FORM_A_FP64: return by_map<0, prngd::kFormA>(map, p, u1, u2, n, out, s);
    case PRNG_FORM_L_ALGO1: return by_map<0, prngd::kFormL>(map, p, u1, u2, n, out, s);
    case PRNG_FORM_C_F32PAIR: return by_map<W, prngd::kFormC>(map, p, u1, u2, n, out, s);
    default: return by_map<W, prngd::kFormB>(map, p, u1, u2, n, out, s);
  }
}

}  // namespace
}  // namespace prngd_host

using namespace prngd_host;

extern "C" int prng_convert_pairs(int w, int form, int mode, const uint32_t* d_u1, const uint32_t* d_u2, uint64_t n,
                                  uint64_t* d_out, void* cuda_stream) {
  if (w < 2 || w > 32) return fail(PRNG_EINVAL, "w = %d is outside [2, 32]", w);
  if (form != PRNG_FORM_A_FP64 && form != PRNG_FORM_B_INTBITS && form != PRNG_FORM_C_F32PAIR &&
      form != PRNG_FORM_L_ALGO1)
    return fail(PRNG_EINVAL, "unknown form %d", form);
  if (mode & ~kAllModes) return fail(PRNG_EINVAL, "unknown mode bits 0x%x", (unsigned)mode);
  if (n == 0) return PRNG_OK;
  if (!d_u1 || !d_u2 || !d_out) return fail(PRNG_EINVAL, "null pointer");
  if (((uintptr_t)d_u1 & 3) || ((uintptr_t)d_u2 & 3) || ((uintptr_t)d_out & 7))
    return fail(PRNG_EINVAL, "d_u1 and d_u2 must be 4-byte and d_out 8-byte aligned");
  prngd::FillParams p;
  memset(&p, 0, sizeof(p));
  p.dc = make_divconst(w);
  p.scale = scale_constant(p.dc);
  p.w = w;
  p.one = 1;
  set_mode_constants(p, w, mode & (PRNG_MODE_EQ5 | PRNG_MODE_ONE_MINUS));
  const int map = map_bits_of(form, mode);
  const cudaStream_t s = (cudaStream_t)cuda_stream;
  cudaError_t e;
  if (w == 32) e = by_form<32>(form, map, p, d_u1, d_u2, n, d_out, s);
  else if (w == 24) e = by_form<24>(form, map, p, d_u1, d_u2, n, d_out, s);
  else e = by_form<0>(form, map, p, d_u1, d_u2, n, d_out, s);
  if (e != cudaSuccess) return fail(PRNG_ECUDA, "convert launch: %s", cudaGetErrorString(e));
  return PRNG_OK;
}
