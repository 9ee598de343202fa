// prngd_noalloc.cu -- prng_fill_f64_host_noalloc: the host-memory fill with its device
// staging in a fixed, file-scope device array instead of memory from cudaMalloc.
//
// Who needs this: callers that cannot allocate device memory when they ask for numbers. One
// example is a process whose device memory already belongs to another allocator, such as a
// framework's caching pool that reserved the whole GPU. Another is a service that fixes its
// memory footprint at start-up and must never hit out-of-memory later. A third is a latency-
// sensitive loop that cannot afford cudaMalloc/cudaFree, which may synchronise the whole
// device. The array below is part of the library image: every GPU that loads the library
// holds it until the process exits.
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "prngd.h"
#include "prngd_internal.h"

namespace {

// Staging for one slice of output values, then one reject count per stream of the slice.
constexpr size_t kValueBytes = PRNG_NOALLOC_VALUE_BYTES;
constexpr uint64_t kMaxSliceStreams = PRNG_NOALLOC_MAX_SLICE_STREAMS;
constexpr size_t kScratchBytes = kValueBytes + kMaxSliceStreams * 8;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {};

// Device address of the array on `dev` (current device), looked up once per device. In host
// code the array's name is only a host-side stand-in; the kernel must get this address.
int scratch_address(int dev, void** out) {
  if (dev < 0 || dev >= kMaxDevices) return prngd_host::fail(PRNG_EINVAL, "device %d out of range", dev);
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
      return prngd_host::fail(PRNG_ECUDA, "cudaGetSymbolAddress(noalloc scratch): %s", cudaGetErrorString(e));
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return PRNG_OK;
}

}  // namespace

extern "C" int prng_fill_f64_host_noalloc(prng_t h, double* host_out, uint64_t per_stream, int form,
                                          uint64_t* host_rejects, void* cuda_stream) {
  using prngd_host::fail;
  if (!h) return fail(PRNG_EINVAL, "null handle");
  if (form != PRNG_FORM_A_FP64 && form != PRNG_FORM_B_INTBITS)
    return fail(PRNG_EINVAL, "prng_fill_f64_host_noalloc takes form A (0) or B (1), got %d", form);
  if (per_stream == 0) return PRNG_OK;
  if (!host_out) return fail(PRNG_EINVAL, "host_out is NULL");
  if (per_stream > kValueBytes / 8)
    return fail(PRNG_EINVAL, "per_stream = %llu exceeds the static scratch limit of %llu outputs per stream",
                (unsigned long long)per_stream, (unsigned long long)(kValueBytes / 8));
  int rc = prngd_host::check_handle_device(h);
  if (rc) return rc;
  void* scratch = nullptr;
  rc = scratch_address(h->device, &scratch);
  if (rc) return rc;
  double* d_values = (double*)scratch;
  uint64_t* d_rej = (uint64_t*)((unsigned char*)scratch + kValueBytes);
  const cudaStream_t s = (cudaStream_t)cuda_stream;
  uint64_t slice = kValueBytes / (per_stream * 8);
  if (slice > kMaxSliceStreams) slice = kMaxSliceStreams;
  if (slice > h->n_streams) slice = h->n_streams;
  cudaError_t e;
  // One buffer, one stream: each slice is generated, then copied out, before the next slice
  // overwrites the array (stream order). Nothing in the array needs to start at zero: the
  // kernel writes every value and every reject count of the slice.
  for (uint64_t s0 = 0; s0 < h->n_streams; s0 += slice) {
    const uint64_t cnt = (h->n_streams - s0 < slice) ? h->n_streams - s0 : slice;
    rc = prngd_host::launch_fill(h, prngd_host::state_at(h, s0), cnt, d_values, per_stream, form,
                                 host_rejects ? d_rej : nullptr, s, true);
    if (!rc) {
      e = cudaMemcpyAsync(host_out + s0 * per_stream, d_values, (size_t)cnt * per_stream * 8, cudaMemcpyDeviceToHost, s);
      if (e != cudaSuccess) rc = fail(PRNG_ECUDA, "copy to host: %s", cudaGetErrorString(e));
    }
    if (!rc && host_rejects) {
      e = cudaMemcpyAsync(host_rejects + s0, d_rej, (size_t)cnt * 8, cudaMemcpyDeviceToHost, s);
      if (e != cudaSuccess) rc = fail(PRNG_ECUDA, "reject copy: %s", cudaGetErrorString(e));
    }
    if (rc) {  // the copies already queued write into host memory: let them end before returning
      cudaStreamSynchronize(s);
      return rc;
    }
  }
  e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return fail(PRNG_ECUDA, "sync: %s", cudaGetErrorString(e));
  return PRNG_OK;
}
