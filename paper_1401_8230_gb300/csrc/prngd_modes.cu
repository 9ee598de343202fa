// prngd_modes.cu -- fill kernels for the Eq. 5 and 1 - z maps and for form L (Algorithm 1
// in FP64), any w: the generic per-output path of prngd_fill.cuh (exact conversion of every
// output, runtime w) with the map as a template parameter; TMA tile stores when the output
// has a tensor map, plain stores otherwise.
#include <cuda.h>
#include <cuda_runtime.h>

#include "prngd_fill.cuh"
#include "prngd_internal.h"
#include "prngd_launch.h"

namespace prngd_host {
namespace {
constexpr int kWarpsPerBlock = 8;
constexpr size_t kTmaSmem = (size_t)kWarpsPerBlock * prngd::kTileBytes + 1024;

template <int FORM, int MAP>
cudaError_t launch_generic(const prngd::FillParams& p, const CUtensorMap* tmap, cudaStream_t s) {
  const uint64_t warps = (p.n_streams + 31) / 32;
  const unsigned blocks = (unsigned)((warps + kWarpsPerBlock - 1) / kWarpsPerBlock);
  if (tmap) {
    auto k = prngd::fill_tma_kernel<0, FORM, 1, MAP>;
    static std::atomic<uint64_t> attr{0};
    const cudaError_t e = prngd::smem_limit_once(k, (int)kTmaSmem, attr);
    if (e != cudaSuccess) return e;
    k<<<blocks, kWarpsPerBlock * 32, kTmaSmem, s>>>(p, *tmap);
  } else {
    prngd::fill_plain_kernel<0, FORM, MAP><<<blocks, kWarpsPerBlock * 32, 0, s>>>(p);
  }
  return cudaGetLastError();
}

template <int FORM>
cudaError_t launch_form_map(const prngd::FillParams& p, int map, const CUtensorMap* tmap, cudaStream_t s) {
  if constexpr (FORM == prngd::kFormA) {  // balanced form A (integer conversion) under a map
    constexpr int E = prngd::kMapEq5, O = prngd::kMapOneMinus, V = prngd::kMapCvt;
    switch (map) {
      case V: return launch_generic<FORM, V>(p, tmap, s);
      case V | E: return launch_generic<FORM, V | E>(p, tmap, s);
      case V | O: return launch_generic<FORM, V | O>(p, tmap, s);
      case V | E | O: return launch_generic<FORM, V | E | O>(p, tmap, s);
      default: break;
    }
  }
  switch (map & ~prngd::kMapCvt) {  // form B's rounding route exists in the pair kernels only
    case 0: return launch_generic<FORM, 0>(p, tmap, s);
    case prngd::kMapEq5: return launch_generic<FORM, prngd::kMapEq5>(p, tmap, s);
    case prngd::kMapOneMinus: return launch_generic<FORM, prngd::kMapOneMinus>(p, tmap, s);
    case prngd::kMapEq5 | prngd::kMapOneMinus:
      return launch_generic<FORM, prngd::kMapEq5 | prngd::kMapOneMinus>(p, tmap, s);
    default: return cudaErrorInvalidValue;
  }
}
}  // namespace

cudaError_t launch_fill_map(const prngd::FillParams& p, int form, int map, const CUtensorMap* tmap, cudaStream_t s) {
  switch (form) {
    case PRNG_FORM_A_FP64: return launch_form_map<prngd::kFormA>(p, map, tmap, s);
    case PRNG_FORM_B_INTBITS: return launch_form_map<prngd::kFormB>(p, map, tmap, s);
    case PRNG_FORM_C_F32PAIR: return launch_form_map<prngd::kFormC>(p, map, tmap, s);
    case PRNG_FORM_L_ALGO1: return launch_form_map<prngd::kFormL>(p, map, tmap, s);
    default: return cudaErrorInvalidValue;
  }
}
}  // namespace prngd_host
