// stitch.cu -- places one shard stream inside a whole-input stream.
//
// Chunks are compressed independently (section 3.3.1), so the records of a
// shard that starts on an index superblock (64 chunks) are byte for byte the
// records of the same chunks in the whole-input stream.  The exchange
// between shards is the exclusive scan of their record bytes (the host
// passes its result as record_base); this kernel then copies the shard's
// table entries, rebases its index entries and copies its records to their
// places.  One launch, grid-stride over the three regions.
#include <cuda_runtime.h>

#include <cstdint>

#include "glz_common.h"

namespace glz {

namespace {

__device__ __forceinline__ uint64_t ld_u64_le(const uint8_t *p) {
  return *reinterpret_cast<const uint64_t *>(p);  // 8-byte aligned, little endian
}

__device__ __forceinline__ uint32_t ld_u32_le(const uint8_t *p) {
  return *reinterpret_cast<const uint32_t *>(p);
}

// The shard header must describe the shard the host named and a chunk size
// that splits the whole input into total_chunks chunks.
__device__ bool shard_header_ok(const StitchArgs &A) {
  const uint8_t *h = A.shard;
  if (ld_u32_le(h) != 0x315A4C47u || (h[4] != 1 && h[4] != 2)) return false;  // "GLZ1", v1/v2
  const uint32_t C = ld_u32_le(h + 12);
  if (C < 16 || C > kMaxChunk || C % 16 != 0) return false;
  const uint64_t nc = ld_u32_le(h + 20), n = ld_u64_le(h + 24);
  if (nc != A.shard_chunks || (n + C - 1) / C != nc) return false;
  return (A.total_bytes + C - 1) / C == A.total_chunks;
}

}  // namespace

__global__ void __launch_bounds__(256) stitch_kernel(StitchArgs A) {
  if (!shard_header_ok(A)) {
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(A.err, kErrCorrupt);
    return;
  }
  const uint64_t tid = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  const uint64_t nthreads = static_cast<uint64_t>(gridDim.x) * blockDim.x;

  // header: the shard's own fields, with the whole input's counts
  if (A.chunk_base == 0 && tid < kHeaderBytes / 4) {
    uint32_t w = ld_u32_le(A.shard + 4 * tid);
    if (tid == 5) w = static_cast<uint32_t>(A.total_chunks);
    if (tid == 6) w = static_cast<uint32_t>(A.total_bytes);
    if (tid == 7) w = static_cast<uint32_t>(A.total_bytes >> 32);
    reinterpret_cast<uint32_t *>(A.out)[tid] = w;
  }

  // table entries
  const uint64_t *tab = reinterpret_cast<const uint64_t *>(A.shard + kHeaderBytes);
  uint64_t *tab_out =
      reinterpret_cast<uint64_t *>(A.out + kHeaderBytes) + A.chunk_base;
  for (uint64_t i = tid; i < A.shard_chunks; i += nthreads) tab_out[i] = tab[i];

  // index entries, rebased to the whole stream's records region
  const uint64_t n_idx = (A.shard_chunks + kIndexStride - 1) / kIndexStride;
  const uint64_t *idx = tab + A.shard_chunks;
  uint64_t *idx_out = reinterpret_cast<uint64_t *>(A.out + kHeaderBytes) +
                      A.total_chunks + A.chunk_base / kIndexStride;
  for (uint64_t i = tid; i < n_idx; i += nthreads) idx_out[i] = idx[i] + A.record_base;

  // records: aligned 32-bit destination words, each assembled from the two
  // aligned source words that cover it (the source start is 8-byte aligned,
  // so its misalignment after the head equals the head length)
  const uint8_t *src = A.shard + A.src_records;
  uint8_t *dst = A.out + A.dst_records;
  const uint64_t n = A.record_bytes;
  const uint64_t head =
      min(n, static_cast<uint64_t>((4u - (reinterpret_cast<uintptr_t>(dst) & 3u)) & 3u));
  if (tid < head) dst[tid] = src[tid];
  const uint64_t words = (n - head) / 4;
  uint32_t *d32 = reinterpret_cast<uint32_t *>(dst + head);
  const uint32_t *s32 = reinterpret_cast<const uint32_t *>(src);  // src + head - head
  if (head == 0) {
    for (uint64_t j = tid; j < words; j += nthreads) d32[j] = s32[j];
  } else {
    const uint32_t sh = 8u * static_cast<uint32_t>(head);
    for (uint64_t j = tid; j < words; j += nthreads)
      d32[j] = __funnelshift_r(s32[j], s32[j + 1], sh);
  }
  const uint64_t done = head + 4 * words;
  if (tid < n - done) dst[done + tid] = src[done + tid];
}

cudaError_t launch_stitch(const StitchArgs &A, int sms, cudaStream_t stream) {
  const uint64_t work = A.record_bytes / 4 + A.shard_chunks + kHeaderBytes;
  uint64_t grid = (work + 255) / 256;
  const uint64_t cap = static_cast<uint64_t>(sms) * 8;
  if (grid > cap) grid = cap;
  if (grid == 0) grid = 1;
  stitch_kernel<<<static_cast<unsigned>(grid), 256, 0, stream>>>(A);
  return cudaGetLastError();
}

}  // namespace glz
