// prngd_launch.h -- host helper shared by the kernel launchers.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

namespace prngd {

// Raise kernel k's dynamic shared-memory limit to `bytes`, once per device: the attribute
// belongs to the device's context, so every device the process launches on needs its own call.
// `done` holds one bit per device (devices from 64 on call every time); safe from several
// host threads.
template <class Kernel>
inline cudaError_t smem_limit_once(Kernel k, int bytes, std::atomic<uint64_t>& done) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const uint64_t bit = (dev >= 0 && dev < 64) ? (1ull << dev) : 0;
  if (bit && (done.load(std::memory_order_acquire) & bit)) return cudaSuccess;
  e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess && bit) done.fetch_or(bit, std::memory_order_release);
  return e;
}

}  // namespace prngd
