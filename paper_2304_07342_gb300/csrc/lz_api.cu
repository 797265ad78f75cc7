// lz_api.cu -- host side of the C ABI declared in include/lz.h: argument
// validation, the context (scratch + sticky error word), shared-memory
// layout and kernel dispatch.  No compression arithmetic runs on the host.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>
#include <mutex>

#include "../../include/lz.h"
#include "glz_common.h"

namespace glz {
cudaError_t launch_compress_s1(const CompressArgs &A, uint32_t nj, int block,
                               unsigned grid, cudaStream_t stream);
cudaError_t launch_compress_s2(const CompressArgs &A, uint32_t nj, int block,
                               unsigned grid, cudaStream_t stream);
cudaError_t launch_compress_s4(const CompressArgs &A, uint32_t nj, int block,
                               unsigned grid, cudaStream_t stream);
cudaError_t launch_decompress(DecompressArgs A, int block, cudaStream_t stream);

// Empty input: the stream is the header alone (n_chunks = 0, n_bytes = 0).
__global__ void header_kernel(uint8_t *out, uint32_t S, uint32_t offB,
                              uint32_t m, uint32_t M, uint32_t C, uint32_t W,
                              unsigned long long *out_bytes) {
  const uint32_t i = threadIdx.x;
  if (i >= kHeaderBytes) return;
  const uint8_t fixed[9] = {'G', 'L', 'Z', '1', 1,
                            static_cast<uint8_t>(S), static_cast<uint8_t>(offB),
                            static_cast<uint8_t>(m), static_cast<uint8_t>(M)};
  uint8_t b = 0;
  if (i < 9) b = fixed[i];
  else if (i >= 12 && i < 16) b = static_cast<uint8_t>(C >> (8 * (i - 12)));
  else if (i >= 16 && i < 20) b = static_cast<uint8_t>(W >> (8 * (i - 16)));
  out[i] = b;
  if (i == 0) *out_bytes = kHeaderBytes;
}

static cudaError_t launch_header(uint8_t *out, uint32_t S, uint32_t offB,
                                 uint32_t m, uint32_t M, uint32_t C, uint32_t W,
                                 unsigned long long *out_bytes,
                                 cudaStream_t stream) {
  header_kernel<<<1, 32, 0, stream>>>(out, S, offB, m, M, C, W, out_bytes);
  return cudaGetLastError();
}
}  // namespace glz

struct lz_ctx {
  int device = 0;
  int smem_optin = 0;       // max dynamic shared memory per block (bytes)
  int smem_per_sm = 0;      // shared memory per multiprocessor (bytes)
  int smem_reserved = 0;    // shared memory the runtime reserves per block
  int sms = 0;              // multiprocessors
  void *scratch = nullptr;  // [0,16): work counter; [16, ...): status words
  size_t scratch_bytes = 0;
  uint32_t *d_err = nullptr;
  std::mutex mu;
};

namespace {

constexpr int kCompressWarps = 4;      // warps per block (fewer if smem-bound)
constexpr uint32_t kParkSlots = 3;     // parked records per compressing warp
constexpr int kDecompressBlock = 256;  // 8 warps, one chunk per warp
constexpr size_t kScratchHead = 16;

uint64_t div_up(uint64_t a, uint64_t b) { return (a + b - 1) / b; }
uint32_t round16(uint64_t v) { return static_cast<uint32_t>((v + 15) & ~15ull); }
uint32_t off_bytes(uint32_t W) { return W <= 256 ? 1u : 2u; }

// Worst-case record of a chunk of k symbols (see lz_compressed_bound).
uint64_t record_bound(uint64_t k, uint32_t S, uint32_t offB, uint32_t m) {
  const uint64_t extra = (1u + offB > S * m) ? (1u + offB - S * m) : 0u;
  return div_up(k, 8) + static_cast<uint64_t>(S) * k + extra * (k / m);
}

bool params_ok(const lz_params *p) {
  if (!p) return false;
  const uint32_t S = p->symbol_bytes, C = p->chunk_bytes, W = p->window;
  if (S != 1 && S != 2 && S != 4) return false;
  if (C < 16 || C > glz::kMaxChunk || C % 16 != 0) return false;
  if (W < 1 || W > glz::kMaxWindow) return false;
  if (p->min_match < 1 || p->min_match > p->max_match || p->max_match > 255)
    return false;
  return true;
}

// Shared-memory slice of one compressing warp.
glz::CompressSmem compress_layout(const lz_params *p) {
  const uint32_t S = p->symbol_bytes, C = p->chunk_bytes;
  const uint32_t k = C / S;
  const uint32_t offB = off_bytes(p->window);
  const uint64_t extra = (1u + offB > S * p->min_match) ? (1u + offB - S * p->min_match) : 0u;
  const uint64_t pay_bytes = static_cast<uint64_t>(S) * k + extra * (k / p->min_match);
  glz::CompressSmem sm{};
  uint32_t at = 0;
  sm.in_off = at;
  at += round16(C);
  sm.prev_off = at;
  at += round16((p->window > 256 ? 2ull : 1ull) * k);
  sm.flags_off = at;
  at += round16(div_up(k, 32) * 4);
  sm.pay_off = at;
  const uint32_t pay_region = round16(pay_bytes + 16);
  sm.pay_bytes = pay_region;
  at += pay_region;
  sm.maybe_off = at;
  at += round16(div_up(k, 32) * 4);
  sm.mbar_off = at;
  at += 16;
  sm.per_warp = (at + 127) & ~127u;
  // hash table of u16 entries inside the payload region, at most 2^15
  uint32_t lg = 1;
  while (lg < 15 && (2u << (lg + 1)) <= pay_region) ++lg;
  sm.hash_log2 = lg;
  return sm;
}

lz_status cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return LZ_OK;
  if (e == cudaErrorMemoryAllocation) return LZ_ERR_NOMEM;
  return LZ_ERR_CUDA;
}

// Make sure the scratch area holds `bytes`; synchronous when it grows.
lz_status reserve_scratch(lz_ctx *ctx, size_t bytes) {
  if (ctx->scratch_bytes >= bytes) return LZ_OK;
  size_t want = ctx->scratch_bytes ? ctx->scratch_bytes : (1u << 16);
  while (want < bytes) want *= 2;
  if (ctx->scratch) {
    cudaError_t e = cudaFree(ctx->scratch);  // waits for work using it
    ctx->scratch = nullptr;
    ctx->scratch_bytes = 0;
    if (e != cudaSuccess) return LZ_ERR_CUDA;
  }
  void *p = nullptr;
  cudaError_t e = cudaMalloc(&p, want);
  if (e != cudaSuccess) return cuda_status(e);
  ctx->scratch = p;
  ctx->scratch_bytes = want;
  return LZ_OK;
}

}  // namespace

extern "C" {

const char *lz_status_string(lz_status s) {
  switch (s) {
    case LZ_OK: return "LZ_OK";
    case LZ_ERR_INVALID_ARG: return "LZ_ERR_INVALID_ARG";
    case LZ_ERR_BUFFER_TOO_SMALL: return "LZ_ERR_BUFFER_TOO_SMALL";
    case LZ_ERR_CORRUPT: return "LZ_ERR_CORRUPT";
    case LZ_ERR_NOMEM: return "LZ_ERR_NOMEM";
    case LZ_ERR_CUDA: return "LZ_ERR_CUDA";
    case LZ_ERR_TIMEOUT: return "LZ_ERR_TIMEOUT";
    case LZ_ERR_INTERNAL: return "LZ_ERR_INTERNAL";
  }
  return "LZ_ERR_UNKNOWN";
}

lz_status lz_check_params(const lz_params *p) {
  return params_ok(p) ? LZ_OK : LZ_ERR_INVALID_ARG;
}

uint64_t lz_compressed_bound(uint64_t n_bytes, const lz_params *p) {
  if (!params_ok(p)) return 0;
  const uint32_t S = p->symbol_bytes, C = p->chunk_bytes;
  const uint32_t offB = off_bytes(p->window);
  const uint64_t nc = div_up(n_bytes, C);
  uint64_t total = glz::kHeaderBytes + glz::kTableEntry * nc +
                   8ull * div_up(nc, glz::kIndexStride);
  if (nc == 0) return total;
  total += (nc - 1) * record_bound(C / S, S, offB, p->min_match);
  total += record_bound((n_bytes - (nc - 1) * C) / S, S, offB, p->min_match);
  return total;
}

lz_status lz_create(lz_ctx **out, int device) {
  if (!out) return LZ_ERR_INVALID_ARG;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess) return LZ_ERR_CUDA;
  if (device < 0 || device >= ndev) return LZ_ERR_INVALID_ARG;
  if (cudaSetDevice(device) != cudaSuccess) return LZ_ERR_CUDA;
  lz_ctx *ctx = new (std::nothrow) lz_ctx();
  if (!ctx) return LZ_ERR_NOMEM;
  ctx->device = device;
  cudaError_t e = cudaDeviceGetAttribute(&ctx->smem_optin,
                                         cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
  if (e == cudaSuccess)
    e = cudaDeviceGetAttribute(&ctx->smem_per_sm,
                               cudaDevAttrMaxSharedMemoryPerMultiprocessor, device);
  if (e == cudaSuccess)
    e = cudaDeviceGetAttribute(&ctx->smem_reserved,
                               cudaDevAttrReservedSharedMemoryPerBlock, device);
  if (e == cudaSuccess)
    e = cudaDeviceGetAttribute(&ctx->sms, cudaDevAttrMultiProcessorCount, device);
  if (e == cudaSuccess) e = cudaMalloc(&ctx->d_err, 256);
  if (e == cudaSuccess) e = cudaMemset(ctx->d_err, 0, 256);
  if (e != cudaSuccess) {
    if (ctx->d_err) cudaFree(ctx->d_err);
    delete ctx;
    return cuda_status(e);
  }
  lz_status s = reserve_scratch(ctx, 1u << 16);
  if (s != LZ_OK) {
    cudaFree(ctx->d_err);
    delete ctx;
    return s;
  }
  *out = ctx;
  return LZ_OK;
}

void lz_destroy(lz_ctx *ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->device);
  cudaDeviceSynchronize();
  if (ctx->scratch) cudaFree(ctx->scratch);
  if (ctx->d_err) cudaFree(ctx->d_err);
  delete ctx;
}

lz_status lz_compress(lz_ctx *ctx, const void *d_in, uint64_t n_bytes,
                      const lz_params *p, void *d_out, uint64_t out_cap,
                      uint64_t *d_out_bytes, lz_stream_t stream) {
  if (!ctx || !params_ok(p) || !d_out || !d_out_bytes) return LZ_ERR_INVALID_ARG;
  if (n_bytes > 0 && !d_in) return LZ_ERR_INVALID_ARG;
  if (reinterpret_cast<uintptr_t>(d_out_bytes) % 8 != 0) return LZ_ERR_INVALID_ARG;
  const uint32_t S = p->symbol_bytes, C = p->chunk_bytes;
  if (n_bytes % S != 0) return LZ_ERR_INVALID_ARG;
  const uint64_t nc = div_up(n_bytes, C);
  if (nc > 0xFFFFFFFFull) return LZ_ERR_INVALID_ARG;
  const uint64_t records_at = glz::kHeaderBytes + glz::kTableEntry * nc +
                              8ull * div_up(nc, glz::kIndexStride);
  if (out_cap < records_at) return LZ_ERR_BUFFER_TOO_SMALL;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  std::lock_guard<std::mutex> lock(ctx->mu);
  if (cudaSetDevice(ctx->device) != cudaSuccess) return LZ_ERR_CUDA;
  const uint32_t offB = off_bytes(p->window);
  auto *out_bytes = reinterpret_cast<unsigned long long *>(d_out_bytes);
  if (nc == 0)
    return cuda_status(glz::launch_header(static_cast<uint8_t *>(d_out), S, offB,
                                          p->min_match, p->max_match, C,
                                          p->window, out_bytes, st));

  glz::CompressSmem sm = compress_layout(p);
  if (static_cast<int64_t>(sm.per_warp) > ctx->smem_optin) return LZ_ERR_INVALID_ARG;
  // warps per block: the choice that keeps the most warps resident under the
  // per-SM shared-memory limit (each block also reserves some shared memory)
  int block = 32;
  int64_t best_warps = 0, best_blocks = 1;
  for (int wpb = 1; wpb <= kCompressWarps; wpb *= 2) {
    const int64_t per_block = static_cast<int64_t>(sm.per_warp) * wpb + ctx->smem_reserved;
    if (per_block - ctx->smem_reserved > ctx->smem_optin) break;
    int64_t blocks = ctx->smem_per_sm / per_block;
    if (blocks > 32) blocks = 32;
    if (blocks * wpb > best_warps) {
      best_warps = blocks * wpb;
      best_blocks = blocks;
      block = 32 * wpb;
    }
  }
  const uint64_t wpb = block / 32;
  uint64_t grid = div_up(nc, wpb);
  if (grid > static_cast<uint64_t>(best_blocks) * ctx->sms) grid = best_blocks * ctx->sms;
  // scratch: work counter, nc status words, parking slots of every warp
  const uint32_t slot_bytes = round16(div_up(C / S, 8) + sm.pay_bytes + 16);
  const size_t status_end = kScratchHead + 8ull * nc;
  const size_t park_at = (status_end + 255) & ~static_cast<size_t>(255);
  const size_t need = park_at + static_cast<size_t>(slot_bytes) * kParkSlots * wpb * grid;
  lz_status s = reserve_scratch(ctx, need);
  if (s != LZ_OK) return s;
  cudaError_t e = cudaMemsetAsync(ctx->scratch, 0, status_end, st);
  if (e != cudaSuccess) return LZ_ERR_CUDA;

  glz::CompressArgs A{};
  A.in = static_cast<const uint8_t *>(d_in);
  A.n = n_bytes;
  A.out = static_cast<uint8_t *>(d_out);
  A.cap = out_cap;
  A.out_bytes = out_bytes;
  A.S = S;
  A.C = C;
  A.W = p->window;
  A.m = p->min_match;
  A.M = p->max_match;
  A.offB = offB;
  A.nc = static_cast<uint32_t>(nc);
  A.records_at = records_at;
  A.in_aligned = (reinterpret_cast<uintptr_t>(d_in) % 16) == 0;
  A.sm = sm;
  A.park = static_cast<uint8_t *>(ctx->scratch) + park_at;
  A.park_slots = kParkSlots;
  A.park_slot_bytes = slot_bytes;
  A.ticket = static_cast<uint32_t *>(ctx->scratch);
  A.status = reinterpret_cast<unsigned long long *>(
      static_cast<uint8_t *>(ctx->scratch) + kScratchHead);
  A.err = ctx->d_err;
  uint32_t nj = 1;
  while (32 * nj < p->window) nj *= 2;
  const unsigned g = static_cast<unsigned>(grid);
  switch (S) {
    case 1: e = glz::launch_compress_s1(A, nj, block, g, st); break;
    case 2: e = glz::launch_compress_s2(A, nj, block, g, st); break;
    default: e = glz::launch_compress_s4(A, nj, block, g, st); break;
  }
  return cuda_status(e);
}

lz_status lz_decompressed_size(const void *d_in, uint64_t in_bytes,
                               uint64_t *h_n, lz_stream_t stream) {
  if (!d_in || !h_n) return LZ_ERR_INVALID_ARG;
  if (in_bytes < glz::kHeaderBytes) return LZ_ERR_CORRUPT;
  uint8_t h[32];
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (cudaMemcpyAsync(h, d_in, 32, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return LZ_ERR_CUDA;
  auto u32 = [&](int at) {
    return static_cast<uint32_t>(h[at]) | (static_cast<uint32_t>(h[at + 1]) << 8) |
           (static_cast<uint32_t>(h[at + 2]) << 16) | (static_cast<uint32_t>(h[at + 3]) << 24);
  };
  uint64_t n = 0;
  for (int i = 0; i < 8; ++i) n |= static_cast<uint64_t>(h[24 + i]) << (8 * i);
  lz_params p{h[5], u32(12), u32(16), h[7], h[8]};
  if (std::memcmp(h, "GLZ1", 4) != 0 || h[4] != 1 || h[9] || h[10] || h[11] ||
      !params_ok(&p) || h[6] != off_bytes(p.window) || n % p.symbol_bytes != 0 ||
      u32(20) != div_up(n, p.chunk_bytes))
    return LZ_ERR_CORRUPT;
  *h_n = n;
  return LZ_OK;
}

lz_status lz_decompress(lz_ctx *ctx, const void *d_in, uint64_t in_bytes,
                        void *d_out, uint64_t out_cap, uint64_t *d_out_bytes,
                        lz_stream_t stream) {
  if (!ctx || !d_in || !d_out_bytes) return LZ_ERR_INVALID_ARG;
  if (reinterpret_cast<uintptr_t>(d_out_bytes) % 8 != 0) return LZ_ERR_INVALID_ARG;
  if (out_cap > 0 && !d_out) return LZ_ERR_INVALID_ARG;
  if (in_bytes < glz::kHeaderBytes) return LZ_ERR_CORRUPT;
  std::lock_guard<std::mutex> lock(ctx->mu);
  if (cudaSetDevice(ctx->device) != cudaSuccess) return LZ_ERR_CUDA;
  glz::DecompressArgs A{};
  A.in = static_cast<const uint8_t *>(d_in);
  A.in_bytes = in_bytes;
  A.out = static_cast<uint8_t *>(d_out);
  A.out_cap = out_cap;
  A.out_bytes = reinterpret_cast<unsigned long long *>(d_out_bytes);
  A.err = ctx->d_err;
  A.out_aligned = (reinterpret_cast<uintptr_t>(d_out) % 16) == 0;
  return cuda_status(glz::launch_decompress(A, kDecompressBlock,
                                            reinterpret_cast<cudaStream_t>(stream)));
}

lz_status lz_sync(lz_ctx *ctx, lz_stream_t stream) {
  if (!ctx) return LZ_ERR_INVALID_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (cudaSetDevice(ctx->device) != cudaSuccess) return LZ_ERR_CUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return LZ_ERR_CUDA;
  uint32_t h = 0;
  if (cudaMemcpyAsync(&h, ctx->d_err, 4, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return LZ_ERR_CUDA;
  if (h == 0) return LZ_OK;
  if (cudaMemsetAsync(ctx->d_err, 0, 4, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return LZ_ERR_CUDA;
  if (h & glz::kErrInternal) return LZ_ERR_INTERNAL;
  if (h & glz::kErrTimeout) return LZ_ERR_TIMEOUT;
  if (h & glz::kErrCorrupt) return LZ_ERR_CORRUPT;
  return LZ_ERR_BUFFER_TOO_SMALL;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Compression that allocates nothing.
//
// Some callers cannot allocate device memory at the point where they need to
// compress: code running inside a custom allocator or an out-of-memory
// handler, a pre-sized real-time pipeline that forbids allocation after
// start-up, or a plug-in whose host only lends it buffers.  For them,
// lz_compress_noalloc takes its scratch (work counter, error word and one
// look-back status word per chunk) from the fixed device array below, which
// every GPU that loads this library holds until the process exits.  It runs
// the regular compression kernel with no parking slots, so a chunk whose
// offset is not known yet waits for its predecessors instead of moving on.

namespace {

constexpr uint32_t kNoAllocMaxChunks = 65536;  // chunks per call, at most
constexpr size_t kNoAllocHead = 16;            // [0,4) counter, [4,8) error word
constexpr size_t kNoAllocBytes = kNoAllocHead + 8ull * kNoAllocMaxChunks;  // 512 KiB + 16

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

// If the call's kernel raised an error other than "output too small" (whose
// needed size is already in *out_bytes), report it as a stream size of 0;
// clear the word for the next call.
__global__ void noalloc_report(uint32_t *err, unsigned long long *out_bytes) {
  if (threadIdx.x == 0 && *err != 0) {
    if (*err & ~glz::kErrSmall) *out_bytes = 0;
    *err = 0;
  }
}

struct NoAllocDevice {
  bool ready = false;
  unsigned char *scratch = nullptr;  // device address of g_noalloc_scratch
  int smem_optin = 0, smem_per_sm = 0, smem_reserved = 0, sms = 0;
};

// Per-device set-up, done once with that device current: the device address
// of the static scratch array (the host-side symbol is only a stand-in) and
// the launch limits.
lz_status noalloc_device(int dev, NoAllocDevice **out) {
  static std::mutex mu;
  static NoAllocDevice devs[64];
  if (dev < 0 || dev >= 64) return LZ_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lock(mu);
  NoAllocDevice &d = devs[dev];
  if (!d.ready) {
    void *ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr)
      return LZ_ERR_CUDA;
    if (cudaDeviceGetAttribute(&d.smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) !=
            cudaSuccess ||
        cudaDeviceGetAttribute(&d.smem_per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor,
                               dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&d.smem_reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev) !=
            cudaSuccess ||
        cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      return LZ_ERR_CUDA;
    d.scratch = static_cast<unsigned char *>(ptr);
    d.ready = true;
  }
  *out = &d;
  return LZ_OK;
}

}  // namespace

extern "C" lz_status lz_compress_noalloc(const void *d_in, uint64_t n_bytes,
                                         const lz_params *p, void *d_out, uint64_t out_cap,
                                         uint64_t *d_out_bytes, lz_stream_t stream) {
  if (!params_ok(p) || !d_out || !d_out_bytes) return LZ_ERR_INVALID_ARG;
  if (n_bytes > 0 && !d_in) return LZ_ERR_INVALID_ARG;
  if (reinterpret_cast<uintptr_t>(d_out_bytes) % 8 != 0) return LZ_ERR_INVALID_ARG;
  const uint32_t S = p->symbol_bytes, C = p->chunk_bytes;
  if (n_bytes % S != 0) return LZ_ERR_INVALID_ARG;
  const uint64_t nc = div_up(n_bytes, C);
  if (nc > kNoAllocMaxChunks) return LZ_ERR_INVALID_ARG;  // beyond the fixed scratch
  const uint64_t records_at = glz::kHeaderBytes + glz::kTableEntry * nc +
                              8ull * div_up(nc, glz::kIndexStride);
  if (out_cap < records_at) return LZ_ERR_BUFFER_TOO_SMALL;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return LZ_ERR_CUDA;
  NoAllocDevice *nd = nullptr;
  lz_status s = noalloc_device(dev, &nd);
  if (s != LZ_OK) return s;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const uint32_t offB = off_bytes(p->window);
  auto *out_bytes = reinterpret_cast<unsigned long long *>(d_out_bytes);
  if (nc == 0)
    return cuda_status(glz::launch_header(static_cast<uint8_t *>(d_out), S, offB,
                                          p->min_match, p->max_match, C, p->window,
                                          out_bytes, st));
  const glz::CompressSmem sm = compress_layout(p);
  if (static_cast<int64_t>(sm.per_warp) > nd->smem_optin) return LZ_ERR_INVALID_ARG;
  int block = 32;
  int64_t best_warps = 0, best_blocks = 1;
  for (int wpb = 1; wpb <= kCompressWarps; wpb *= 2) {
    const int64_t per_block = static_cast<int64_t>(sm.per_warp) * wpb + nd->smem_reserved;
    if (per_block - nd->smem_reserved > nd->smem_optin) break;
    int64_t blocks = nd->smem_per_sm / per_block;
    if (blocks > 32) blocks = 32;
    if (blocks * wpb > best_warps) {
      best_warps = blocks * wpb;
      best_blocks = blocks;
      block = 32 * wpb;
    }
  }
  uint64_t grid = div_up(nc, block / 32);
  if (grid > static_cast<uint64_t>(best_blocks) * nd->sms) grid = best_blocks * nd->sms;
  // the counter and the status words must start at zero; the error word is
  // cleared by the previous call's report (and starts at zero)
  if (cudaMemsetAsync(nd->scratch + kNoAllocHead, 0, 8ull * nc, st) != cudaSuccess ||
      cudaMemsetAsync(nd->scratch, 0, 4, st) != cudaSuccess)
    return LZ_ERR_CUDA;
  glz::CompressArgs A{};
  A.in = static_cast<const uint8_t *>(d_in);
  A.n = n_bytes;
  A.out = static_cast<uint8_t *>(d_out);
  A.cap = out_cap;
  A.out_bytes = out_bytes;
  A.S = S;
  A.C = C;
  A.W = p->window;
  A.m = p->min_match;
  A.M = p->max_match;
  A.offB = offB;
  A.nc = static_cast<uint32_t>(nc);
  A.records_at = records_at;
  A.in_aligned = (reinterpret_cast<uintptr_t>(d_in) % 16) == 0;
  A.sm = sm;
  A.park = nullptr;  // no parking slots: blocking look-back
  A.park_slots = 0;
  A.park_slot_bytes = 0;
  A.ticket = reinterpret_cast<uint32_t *>(nd->scratch);
  A.err = reinterpret_cast<uint32_t *>(nd->scratch + 4);
  A.status = reinterpret_cast<unsigned long long *>(nd->scratch + kNoAllocHead);
  uint32_t nj = 1;
  while (32 * nj < p->window) nj *= 2;
  cudaError_t e;
  const unsigned g = static_cast<unsigned>(grid);
  switch (S) {
    case 1: e = glz::launch_compress_s1(A, nj, block, g, st); break;
    case 2: e = glz::launch_compress_s2(A, nj, block, g, st); break;
    default: e = glz::launch_compress_s4(A, nj, block, g, st); break;
  }
  if (e != cudaSuccess) return cuda_status(e);
  noalloc_report<<<1, 32, 0, st>>>(A.err, out_bytes);
  return cuda_status(cudaGetLastError());
}
