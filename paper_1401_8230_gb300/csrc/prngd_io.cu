// prngd_io.cu -- fills into host memory: generate slices of streams on the device and copy
// each slice to the host while the next one is generated (two CUDA streams, two buffers).
#include <cuda_runtime.h>
#include <stdint.h>

#include "prngd.h"
#include "prngd_internal.h"

namespace prngd_host {

static constexpr size_t kSliceBytes = (size_t)256 << 20;

void release_aux(prng_ctx* h) {
  for (int b = 0; b < 2; ++b) {
    if (h->d_stage[b]) cudaFree(h->d_stage[b]);
    if (h->io_stream[b]) cudaStreamDestroy(h->io_stream[b]);
    h->d_stage[b] = nullptr;
    h->io_stream[b] = nullptr;
  }
  if (h->d_rej_stage) cudaFree(h->d_rej_stage);
  h->d_rej_stage = nullptr;
  h->stage_bytes = 0;
}

// Pinned and pageable destinations take the same route: slices generated on the device, each
// copied by the copy engines while the next is generated. Into pinned memory the copy is a
// direct DMA at the host link's rate (measured 0.995 of a plain device-to-host copy); a kernel
// writing the pinned buffer itself over the link was as fast on most boxes but fell to half on
// one, where the copy engines kept the full rate, and it holds the SMs for the whole transfer.
int host_fill(prng_ctx* h, double* host_out, uint64_t per_stream, int form, uint64_t* host_rejects) {
  const size_t row = (size_t)per_stream * 8;
  uint64_t slice = kSliceBytes / row;
  if (slice == 0) slice = 1;
  if (slice > h->n_streams) slice = h->n_streams;
  const size_t need = (size_t)slice * row;
  cudaError_t e = cudaSuccess;
  if (h->stage_bytes < need) {
    for (int b = 0; b < 2; ++b) {
      if (h->d_stage[b]) cudaFree(h->d_stage[b]);
      h->d_stage[b] = nullptr;
    }
    h->stage_bytes = 0;
    for (int b = 0; b < 2; ++b) {
      e = cudaMalloc(&h->d_stage[b], need);
      if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(PRNG_ENOMEM, "staging cudaMalloc(%zu): %s", need, cudaGetErrorString(e));
      }
    }
    h->stage_bytes = need;
  }
  for (int b = 0; b < 2; ++b)
    if (!h->io_stream[b]) {
      e = cudaStreamCreateWithFlags(&h->io_stream[b], cudaStreamNonBlocking);
      if (e != cudaSuccess) return fail(PRNG_ECUDA, "cudaStreamCreate: %s", cudaGetErrorString(e));
    }
  if (host_rejects && !h->d_rej_stage) {
    e = cudaMalloc(&h->d_rej_stage, h->n_streams * 8);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(PRNG_ENOMEM, "reject staging: %s", cudaGetErrorString(e));
    }
  }
  // Work already queued on this handle (other streams) must finish first.
  e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return fail(PRNG_ECUDA, "sync: %s", cudaGetErrorString(e));
  int k = 0;
  for (uint64_t s0 = 0; s0 < h->n_streams; s0 += slice, ++k) {
    const uint64_t cnt = (h->n_streams - s0 < slice) ? h->n_streams - s0 : slice;
    const int b = k & 1;
    int rc = launch_fill(h, state_at(h, s0), cnt, h->d_stage[b], per_stream, form,
                         host_rejects ? h->d_rej_stage + s0 : nullptr, h->io_stream[b], true);
    if (!rc) {
      e = cudaMemcpyAsync(host_out + s0 * per_stream, h->d_stage[b], (size_t)cnt * row, cudaMemcpyDeviceToHost,
                          h->io_stream[b]);
      if (e != cudaSuccess) rc = fail(PRNG_ECUDA, "copy to host: %s", cudaGetErrorString(e));
    }
    if (rc) {  // the copies already queued write into host_out: let them end before returning
      for (int q = 0; q < 2; ++q) cudaStreamSynchronize(h->io_stream[q]);
      return rc;
    }
  }
  for (int b = 0; b < 2; ++b) {
    e = cudaStreamSynchronize(h->io_stream[b]);
    if (e != cudaSuccess) return fail(PRNG_ECUDA, "sync: %s", cudaGetErrorString(e));
  }
  if (host_rejects) {
    e = cudaMemcpy(host_rejects, h->d_rej_stage, h->n_streams * 8, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return fail(PRNG_ECUDA, "reject copy: %s", cudaGetErrorString(e));
  }
  return PRNG_OK;
}

}  // namespace prngd_host
