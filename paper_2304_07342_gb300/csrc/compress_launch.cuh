// compress_launch.cuh -- host-side launch of compress_kernel<S, NJ>:
// dynamic shared-memory opt-in, occupancy-sized persistent grid.
#pragma once

#include <cuda_runtime.h>

#include "compress_impl.cuh"
#include "launch_cache.cuh"

namespace glz {

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
