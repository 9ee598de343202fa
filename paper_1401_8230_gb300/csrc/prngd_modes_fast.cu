// prngd_modes_fast.cu -- fill kernels for the Eq. 5 and 1 - z maps (Section 2) at w = 32 and
// w = 24, forms B and C, and form B's balanced route: the pair fast paths of
// prngd_fill.cuh with the map as a template parameter, TMA tile stores. Separate from prngd.cu so the instantiations compile in parallel.
#include <cuda.h>
#include <cuda_runtime.h>

#include "prngd_fill.cuh"
#include "prngd_internal.h"
#include "prngd_launch.h"

namespace prngd_host {
namespace {
constexpr int kWarpsPerBlock = 8;
constexpr size_t kTmaSmem = (size_t)kWarpsPerBlock * prngd::kTileBytes + 1024;

template <int W, int FORM, int MAP, bool SHIFT>
cudaError_t launch_fast_k(const prngd::FillParams& p, const CUtensorMap* tmap, cudaStream_t s) {
  const uint64_t warps = (p.n_streams + 31) / 32;
  const unsigned blocks = (unsigned)((warps + kWarpsPerBlock - 1) / kWarpsPerBlock);
  auto k = prngd::fill_tma_kernel<W, FORM, 1, MAP, SHIFT>;
  static std::atomic<uint64_t> attr{0};
  const cudaError_t e = prngd::smem_limit_once(k, (int)kTmaSmem, attr);
  if (e != cudaSuccess) return e;
  k<<<blocks, kWarpsPerBlock * 32, kTmaSmem, s>>>(p, *tmap);
  return cudaGetLastError();
}

// shift: the map starts 2 outputs into each row (rows 16 bytes into a 32-byte sector)
template <int W, int FORM, int MAP>
cudaError_t launch_fast(const prngd::FillParams& p, const CUtensorMap* tmap, cudaStream_t s, bool shift) {
  return shift ? launch_fast_k<W, FORM, MAP, true>(p, tmap, s) : launch_fast_k<W, FORM, MAP, false>(p, tmap, s);
}

template <int W, int FORM>
cudaError_t launch_map(const prngd::FillParams& p, int map, const CUtensorMap* tmap, cudaStream_t s, bool shift) {
  constexpr int E = prngd::kMapEq5, O = prngd::kMapOneMinus, V = prngd::kMapCvt;
  switch (map) {
    case E: return launch_fast<W, FORM, E>(p, tmap, s, shift);
    case O: return launch_fast<W, FORM, O>(p, tmap, s, shift);
    case E | O: return launch_fast<W, FORM, E | O>(p, tmap, s, shift);
    default: break;
  }
  if constexpr (FORM == prngd::kFormB) {  // form B's balanced route
    switch (map) {
      case V: return launch_fast<W, FORM, V>(p, tmap, s, shift);
      case V | E: return launch_fast<W, FORM, V | E>(p, tmap, s, shift);
      case V | O: return launch_fast<W, FORM, V | O>(p, tmap, s, shift);
      case V | E | O: return launch_fast<W, FORM, V | E | O>(p, tmap, s, shift);
      default: break;
    }
  }
  return cudaErrorInvalidValue;
}
}  // namespace

cudaError_t launch_fill_map_fast(const prngd::FillParams& p, int form, int map, const CUtensorMap* tmap,
                                 cudaStream_t s, bool shift) {
  if (!tmap) return cudaErrorInvalidValue;
  const bool c = form == PRNG_FORM_C_F32PAIR;
  if (p.w == 32)
    return c ? launch_map<32, prngd::kFormC>(p, map, tmap, s, shift) : launch_map<32, prngd::kFormB>(p, map, tmap, s, shift);
  if (p.w == 24)
    return c ? launch_map<24, prngd::kFormC>(p, map, tmap, s, shift) : launch_map<24, prngd::kFormB>(p, map, tmap, s, shift);
  return cudaErrorInvalidValue;
}
}  // namespace prngd_host
