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

// Pinned (device-mapped) destination: one launch writes straight into host memory over the
// host link with plain coalesced stores; no staging and no copy engine.
static int host_fill_direct(prng_ctx* h, void* dev_out, uint64_t per_stream, int form, uint64_t* host_rejects) {
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return fail(PRNG_ECUDA, "sync: %s", cudaGetErrorString(e));
  if (host_rejects && !h->d_rej_stage) {
    e = cudaMalloc(&h->d_rej_stage, h->n_streams * 8);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(PRNG_ENOMEM, "reject staging: %s", cudaGetErrorString(e));
    }
  }
  int rc = launch_fill(h, h->d_state, h->n_streams, dev_out, per_stream, form, host_rejects ? h->d_rej_stage : nullptr,
                       0, false);
  if (rc) return rc;
  e = cudaStreamSynchronize(0);
  if (e != cudaSuccess) return fail(PRNG_ECUDA, "sync: %s", cudaGetErrorString(e));
  if (host_rejects) {
    e = cudaMemcpy(host_rejects, h->d_rej_stage, h->n_streams * 8, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return fail(PRNG_ECUDA, "reject copy: %s", cudaGetErrorString(e));
  }
  return PRNG_OK;
}

int host_fill(prng_ctx* h, double* host_out, uint64_t per_stream, int form, uint64_t* host_rejects) {
  void* dev_out = nullptr;
  if (device_mapped_host(host_out, &dev_out) && !(((uintptr_t)dev_out) & 7))
    return host_fill_direct(h, dev_out, per_stream, form, host_rejects);
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
    if (rc) return rc;
    e = cudaMemcpyAsync(host_out + s0 * per_stream, h->d_stage[b], (size_t)cnt * row, cudaMemcpyDeviceToHost,
                        h->io_stream[b]);
    if (e != cudaSuccess) return fail(PRNG_ECUDA, "copy to host: %s", cudaGetErrorString(e));
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
