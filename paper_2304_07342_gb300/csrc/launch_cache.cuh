// launch_cache.cuh -- per-device cache of a kernel's launch shape: the
// dynamic shared-memory opt-in and the resident blocks per SM.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <mutex>

namespace glz {

// Launch-shape cache for one kernel instance, one entry per device: the
// shared-memory opt-in (cudaFuncSetAttribute acts on the current device's
// context only) and the occupancy query are redone whenever the block or
// shared-memory size changes on that device.
constexpr int kMaxDevices = 64;

struct LaunchCache {
  struct Entry {
    int block = -1, per_sm = 0, sms = 0;
    size_t smem = 0;
  };
  std::mutex mu;
  Entry dev[kMaxDevices];
};

// Blocks of `kern` resident per SM on the current device for this block and
// smem size.
template <typename K>
static cudaError_t resident_blocks(LaunchCache &lc, K kern, int block,
                                   size_t smem, int *per_sm, int *sms) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(lc.mu);
  LaunchCache::Entry &c = lc.dev[dev];
  if (c.block == block && c.smem == smem) {
    *per_sm = c.per_sm;
    *sms = c.sms;
    return cudaSuccess;
  }
  e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, kern, block, smem);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  c.block = block;
  c.smem = smem;
  c.per_sm = *per_sm;
  c.sms = *sms;
  return cudaSuccess;
}

}  // namespace glz
