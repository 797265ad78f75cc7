// compress_batch.cu -- one persistent launch over the chunks of many buffers
// (each with its own parameters), plus the headers of empty buffers.
#include "compress_launch.cuh"

namespace glz {

// Empty buffers: their stream is the header alone.
__global__ void batch_empty_headers(const BufDesc *empties, uint32_t n) {
  const uint32_t lane = threadIdx.x & 31;
  for (uint32_t i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < n;
       i += gridDim.x * (blockDim.x >> 5)) {
    const BufDesc B = empties[i];
    write_header(B, lane);
    if (lane == 0) *B.out_bytes = kHeaderBytes;
  }
}

template <int NJ>
static cudaError_t launch_batch_nj(const CompressArgs &A, int block, unsigned grid_req,
                                   cudaStream_t stream) {
  auto kern = compress_batch_kernel<NJ>;
  const size_t smem = static_cast<size_t>(A.sm.per_warp) * (block / 32);
  static LaunchCache lc;
  int per_sm = 0, sms = 0;
  cudaError_t e = resident_blocks(lc, kern, block, smem, &per_sm, &sms);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  const uint64_t cap = static_cast<uint64_t>(per_sm) * sms;
  const unsigned grid = static_cast<unsigned>(grid_req < cap ? grid_req : cap);
  kern<<<grid, block, smem, stream>>>(A);
  return cudaGetLastError();
}

cudaError_t launch_compress_batch(const CompressArgs &A, const BufDesc *empties,
                                  uint32_t n_empty, uint32_t nj, int block, unsigned grid,
                                  cudaStream_t stream) {
  if (n_empty) {
    batch_empty_headers<<<(n_empty + 7) / 8, 256, 0, stream>>>(empties, n_empty);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  if (A.total_chunks == 0) return cudaSuccess;
  switch (nj) {
    case 1: return launch_batch_nj<1>(A, block, grid, stream);
    case 2: return launch_batch_nj<2>(A, block, grid, stream);
    case 4: return launch_batch_nj<4>(A, block, grid, stream);
    case 8: return launch_batch_nj<8>(A, block, grid, stream);
    case 16: return launch_batch_nj<16>(A, block, grid, stream);
    case 32: return launch_batch_nj<32>(A, block, grid, stream);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace glz
