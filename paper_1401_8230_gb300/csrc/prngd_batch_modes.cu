// prngd_batch_modes.cu -- the batch kernel for batches whose requests use the Eq. 5 map, 1 - z
// or form L (Section 2 of Demchik and Gulov; Eq. 5 and 6, Algorithm 1): every item calls the
// out-of-line code of its request's (form, map). The build compiles this file once per w
// (PRNGD_ANY_MODE_W = 32, 24, or 0 for the generic code), so the sixteen item variants of each
// w compile in parallel.
#include <cuda_runtime.h>

#include "prngd.h"
#include "prngd_batch.cuh"
#include "prngd_internal.h"

#ifndef PRNGD_ANY_MODE_W
#define PRNGD_ANY_MODE_W 32
#endif

namespace prngd_host {

template <>
cudaError_t launch_batch_any_mode_w<PRNGD_ANY_MODE_W>(const prngd::BatchParams& p, const BatchShape& sh,
                                                       unsigned blocks, int max_req, cudaStream_t s) {
  return prngd::launch_batch_kernel<PRNGD_ANY_MODE_W, prngd::kAnyMode>(p, sh.warps_per_block, blocks, max_req, s);
}

}  // namespace prngd_host
