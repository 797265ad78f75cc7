// compress_launch.cuh -- host-side launch of compress_kernel<S, NJ>:
// dynamic shared-memory opt-in, occupancy-sized persistent grid.
#pragma once

#include <cuda_runtime.h>

#include <mutex>

#include "compress_impl.cuh"

namespace glz {

// Launch-shape cache for one kernel instance (the smem opt-in and the
// occupancy query are done once per block/smem combination).
struct LaunchCache {
  std::mutex mu;
  int block = -1, per_sm = 0, sms = 0;
  size_t smem = 0;
};

// Blocks of `kern` resident per SM for this block and smem size.
template <typename K>
static cudaError_t resident_blocks(LaunchCache &lc, K kern, int block,
                                   size_t smem, int *per_sm, int *sms) {
  std::lock_guard<std::mutex> lock(lc.mu);
  if (lc.block == block && lc.smem == smem) {
    *per_sm = lc.per_sm;
    *sms = lc.sms;
    return cudaSuccess;
  }
  cudaError_t e = cudaFuncSetAttribute(
      kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, kern, block, smem);
  if (e != cudaSuccess) return e;
  int dev = 0;
  e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  lc.block = block;
  lc.smem = smem;
  lc.per_sm = *per_sm;
  lc.sms = *sms;
  return cudaSuccess;
}

template <int S, int NJ>
static cudaError_t launch_compress_nj(const CompressArgs &A, int block, unsigned grid_req,
                                      cudaStream_t stream) {
  auto kern = compress_kernel<S, NJ>;
  const size_t smem = static_cast<size_t>(A.sm.per_warp) * (block / 32);
  static LaunchCache lc;
  int per_sm = 0, sms = 0;
  cudaError_t e = resident_blocks(lc, kern, block, smem, &per_sm, &sms);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  // never more blocks than can be resident (the grid is persistent), never
  // more than the parking slots were sized for
  const uint64_t cap = static_cast<uint64_t>(per_sm) * sms;
  const unsigned grid = static_cast<unsigned>(grid_req < cap ? grid_req : cap);
  kern<<<grid, block, smem, stream>>>(A);
  return cudaGetLastError();
}

template <int S>
static cudaError_t launch_compress_t(const CompressArgs &A, uint32_t nj,
                                     int block, unsigned grid, cudaStream_t stream) {
  switch (nj) {
    case 1: return launch_compress_nj<S, 1>(A, block, grid, stream);
    case 2: return launch_compress_nj<S, 2>(A, block, grid, stream);
    case 4: return launch_compress_nj<S, 4>(A, block, grid, stream);
    case 8: return launch_compress_nj<S, 8>(A, block, grid, stream);
    case 16: return launch_compress_nj<S, 16>(A, block, grid, stream);
    case 32: return launch_compress_nj<S, 32>(A, block, grid, stream);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace glz
