// compress_s4.cu -- instantiations of the compression kernel for
// 4-byte symbols (one translation unit per symbol size so that the
// variants compile in parallel).
#include "compress_launch.cuh"

namespace glz {
cudaError_t launch_compress_s4(const CompressArgs &A, uint32_t nj, int block,
                               unsigned grid, cudaStream_t stream) {
  return launch_compress_t<4>(A, nj, block, grid, stream);
}
}  // namespace glz
