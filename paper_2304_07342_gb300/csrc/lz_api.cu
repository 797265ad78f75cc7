// lz_api.cu -- host side of the C ABI declared in include/lz.h: argument
// validation, the context (scratch + sticky error word), shared-memory
// layout and kernel dispatch.  No compression arithmetic runs on the host.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>
#include <algorithm>
#include <mutex>
#include <new>
#include <vector>

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
cudaError_t launch_compress_batch(const CompressArgs &A, const BufDesc *empties,
                                  uint32_t n_empty, uint32_t nj, int block, unsigned grid,
                                  cudaStream_t stream);
cudaError_t launch_decompress_batch(DecompressBatchArgs B, int block, cudaStream_t stream);
cudaError_t launch_stitch(const StitchArgs &A, int sms, cudaStream_t stream);
cudaError_t launch_huff_compress(const uint8_t *in, uint64_t n, uint8_t *out, uint64_t out_cap,
                                 unsigned long long *out_bytes, unsigned long long *hist,
                                 uint32_t *book, uint32_t *err, int sms, cudaStream_t st);
cudaError_t launch_huff_decompress(const uint8_t *in, uint64_t in_bytes, uint8_t *out,
                                   uint64_t out_cap, unsigned long long *out_bytes,
                                   uint32_t *err, int sms, cudaStream_t st);
uint64_t huff_layout_bits_at(uint64_t n);

// Gather the 32-byte headers of n streams into one device array.
__global__ void gather_headers(const uint8_t *const *ins, const uint64_t *in_bytes,
                               uint32_t n, uint8_t *hdr) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n * 32;
       i += gridDim.x * blockDim.x) {
    const uint32_t item = i / 32, b = i % 32;
    hdr[i] = in_bytes[item] >= 32 ? ins[item][b] : 0;
  }
}

// Empty input: the stream is the header alone (n_chunks = 0, n_bytes = 0).
__global__ void header_kernel(uint8_t *out, uint32_t version, uint32_t S, uint32_t offB,
                              uint32_t m, uint32_t M, uint32_t C, uint32_t W,
                              unsigned long long *out_bytes) {
  const uint32_t i = threadIdx.x;
  if (i >= kHeaderBytes) return;
  const uint8_t fixed[9] = {'G', 'L', 'Z', '1', static_cast<uint8_t>(version),
                            static_cast<uint8_t>(S), static_cast<uint8_t>(offB),
                            static_cast<uint8_t>(m), static_cast<uint8_t>(M)};
  uint8_t b = 0;
  if (i < 9) b = fixed[i];
  else if (i >= 12 && i < 16) b = static_cast<uint8_t>(C >> (8 * (i - 12)));
  else if (i >= 16 && i < 20) b = static_cast<uint8_t>(W >> (8 * (i - 16)));
  out[i] = b;
  if (i == 0) *out_bytes = kHeaderBytes;
}

static cudaError_t launch_header(uint8_t *out, uint32_t version, uint32_t S, uint32_t offB,
                                 uint32_t m, uint32_t M, uint32_t C, uint32_t W,
                                 unsigned long long *out_bytes,
                                 cudaStream_t stream) {
  header_kernel<<<1, 32, 0, stream>>>(out, version, S, offB, m, M, C, W, out_bytes);
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
  lz_test_hooks hooks{};    // test hooks (lz_set_test_hooks); all zero normally
  // lz_compress_host: copy-in, compression and copy-out streams, events,
  // device memory (the input, a size word, the stream) and pinned host
  // words (the look-back word of each piece's last chunk)
  cudaStream_t hs[3] = {nullptr, nullptr, nullptr};
  cudaEvent_t hev[17] = {};
  void *hdev = nullptr;
  size_t hdev_bytes = 0;
  uint64_t *hpin = nullptr;
};

namespace {

constexpr int kCompressWarps = 4;      // warps per block (fewer if smem-bound)
constexpr uint32_t kParkSlots = 3;     // parked records per compressing warp
constexpr int kDecompressBlock = 1024;  // up to 32 warps, one chunk per warp at a time
constexpr size_t kScratchHead = 16;
// The look-back word of a placed chunk (written by the compression kernel):
// bit 63 set, the inclusive prefix of the record bytes in the low 62 bits.
constexpr uint64_t kStatusPrefix = 1ull << 63, kStatusValue = (1ull << 62) - 1;
// lz_compress_host: pieces queued on the GPU ahead of the one whose records
// the host copies out next (less than the 8 event and word slots)
constexpr size_t kHostLag = 6;
// Chunks per compression launch: the warps take chunks from a 32-bit work
// counter and each takes one ticket past the last chunk, so the counter must
// not wrap; the margin covers 2^20 warps.
constexpr uint64_t kMaxLaunchChunks = 0xFFFFFFFFull - (1ull << 20);

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
  // The payload area holds the hash table while the chains are built, then
  // the pointer list of the walk (1 + offB bytes per pointer, at most k / m
  // of them); records are emitted in place or at their destination.  For 1-
  // and 2-byte symbols it takes a table of a quarter as many buckets as the
  // chunk has positions (or the list, if larger): less shared memory per
  // warp, more warps resident.
  // For 4-byte symbols it keeps the size of a worst-case payload, which the
  // literal pre-check's Bloom filter uses (with links and flags) to hold
  // about 10 bits per position.
  uint32_t pay_region = round16(pay_bytes + 16);
  if (S <= 2) {
    uint32_t lgk = 1;
    while ((1u << lgk) < k) ++lgk;
    const uint32_t lgt = lgk > 6 ? lgk - 2 : 4;
    const uint64_t list = (1ull + offB) * (k / p->min_match);
    const uint64_t table = 2ull << lgt;
    pay_region = round16((list > table ? list : table) + 16);
  }
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

// Warps per compression block and resident blocks per SM for a per-warp
// slice of `per_warp` bytes: `want` warps per block (1, 2, 4 or 8) when
// given, else the choice among 1, 2, 4 that keeps the most warps resident
// under the per-SM shared-memory limit (each block also reserves some).
// False when not even one block fits.
bool block_shape(int64_t per_warp, int smem_per_sm, int smem_reserved, int smem_optin,
                 uint32_t want, int *block, int64_t *blocks_per_sm) {
  int64_t best_warps = 0;
  for (int wpb = 1; wpb <= 8; wpb *= 2) {
    if (want ? static_cast<uint32_t>(wpb) != want : wpb > kCompressWarps) continue;
    const int64_t per_block = per_warp * wpb + smem_reserved;
    if (per_block - smem_reserved > smem_optin) break;
    int64_t blocks = smem_per_sm / per_block;
    if (blocks > 32) blocks = 32;
    if (blocks >= 1 && blocks * wpb > best_warps) {
      best_warps = blocks * wpb;
      *blocks_per_sm = blocks;
      *block = 32 * wpb;
    }
  }
  return best_warps > 0;
}

lz_status cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return LZ_OK;
  if (e == cudaErrorMemoryAllocation) return LZ_ERR_NOMEM;
  return LZ_ERR_CUDA;
}

// Shared memory of one decoding block: one block per SM, all of the SM's
// shared memory that a block may take.
uint32_t decode_block_smem(const lz_ctx *ctx) {
  const int64_t per_sm = static_cast<int64_t>(ctx->smem_per_sm) - ctx->smem_reserved;
  return static_cast<uint32_t>(std::min<int64_t>(ctx->smem_optin, per_sm));
}

// Make sure the scratch area holds `bytes`; synchronous when it grows.
lz_status reserve_scratch(lz_ctx *ctx, size_t bytes) {
  if (ctx->scratch_bytes >= bytes) return LZ_OK;
  if (ctx->hooks.fail_alloc) return LZ_ERR_NOMEM;  // injected failure (test hook)
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

lz_status compress_locked(lz_ctx *ctx, const void *d_in, uint64_t n_bytes, const lz_params *p,
                          uint32_t match, uint32_t version, void *d_out, uint64_t out_cap,
                          unsigned long long *out_bytes, cudaStream_t st, uint64_t c0 = 0,
                          uint64_t c1 = ~0ull, bool clear_status = true,
                          uint32_t warps_per_block = 0);

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

lz_status lz_set_test_hooks(lz_ctx *ctx, const lz_test_hooks *hooks) {
  if (!ctx) return LZ_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lock(ctx->mu);
  ctx->hooks = hooks ? *hooks : lz_test_hooks{};
  return LZ_OK;
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
  const uint64_t last = n_bytes - (nc - 1) * C;
  total += record_bound(last / S, S, offB, p->min_match) + last % S;  // a tail adds itself
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
  for (cudaStream_t &h : ctx->hs)
    if (h) cudaStreamDestroy(h);
  for (cudaEvent_t &e : ctx->hev)
    if (e) cudaEventDestroy(e);
  if (ctx->hdev) cudaFree(ctx->hdev);
  if (ctx->hpin) cudaFreeHost(ctx->hpin);
  if (ctx->scratch) cudaFree(ctx->scratch);
  if (ctx->d_err) cudaFree(ctx->d_err);
  delete ctx;
}

lz_status lz_compress(lz_ctx *ctx, const void *d_in, uint64_t n_bytes,
                      const lz_params *p, void *d_out, uint64_t out_cap,
                      uint64_t *d_out_bytes, lz_stream_t stream) {
  return lz_compress_ex(ctx, d_in, n_bytes, p, nullptr, d_out, out_cap, d_out_bytes, stream);
}

lz_status lz_compress_ex(lz_ctx *ctx, const void *d_in, uint64_t n_bytes,
                         const lz_params *p, const lz_options *opt, void *d_out,
                         uint64_t out_cap, uint64_t *d_out_bytes, lz_stream_t stream) {
  if (!ctx || !params_ok(p) || !d_out || !d_out_bytes) return LZ_ERR_INVALID_ARG;
  const uint32_t match = opt ? opt->match : LZ_MATCH_EXACT;
  const uint32_t version = opt && opt->version ? opt->version : 1u;
  if (match != LZ_MATCH_EXACT && match != LZ_MATCH_PAPER && match != LZ_MATCH_OVERLAP)
    return LZ_ERR_INVALID_ARG;
  if (version != 1 && version != 2) return LZ_ERR_INVALID_ARG;
  if (match == LZ_MATCH_OVERLAP && version != 2) return LZ_ERR_INVALID_ARG;
  if (opt && opt->warps_per_block && opt->warps_per_block != 1 && opt->warps_per_block != 2 &&
      opt->warps_per_block != 4 && opt->warps_per_block != 8)
    return LZ_ERR_INVALID_ARG;
  if (n_bytes > 0 && !d_in) return LZ_ERR_INVALID_ARG;
  if (reinterpret_cast<uintptr_t>(d_out_bytes) % 8 != 0) return LZ_ERR_INVALID_ARG;
  const uint32_t S = p->symbol_bytes, C = p->chunk_bytes;
  if (version == 1 && n_bytes % S != 0) return LZ_ERR_INVALID_ARG;  // tails: version 2
  const uint64_t nc = div_up(n_bytes, C);
  if (nc > kMaxLaunchChunks) return LZ_ERR_INVALID_ARG;
  const uint64_t records_at = glz::kHeaderBytes + glz::kTableEntry * nc +
                              8ull * div_up(nc, glz::kIndexStride);
  if (out_cap < records_at) return LZ_ERR_BUFFER_TOO_SMALL;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  std::lock_guard<std::mutex> lock(ctx->mu);
  if (cudaSetDevice(ctx->device) != cudaSuccess) return LZ_ERR_CUDA;
  return compress_locked(ctx, d_in, n_bytes, p, match, version, d_out, out_cap,
                         reinterpret_cast<unsigned long long *>(d_out_bytes), st, 0, ~0ull, true,
                         opt ? opt->warps_per_block : 0u);
}

}  // extern "C"

namespace {

// Enqueue one compression whose arguments lz_compress_ex has checked, with
// the context's lock held and its device current: chunks [c0, c1) of the
// buffer (all of them by default).  The look-back status words of every
// chunk of the buffer are cleared when clear_status is set; a launch over
// a later range of the same buffer keeps them (the ranges before it have
// published their prefixes) and clears only the work counter.
lz_status compress_locked(lz_ctx *ctx, const void *d_in, uint64_t n_bytes, const lz_params *p,
                          uint32_t match, uint32_t version, void *d_out, uint64_t out_cap,
                          unsigned long long *out_bytes, cudaStream_t st, uint64_t c0,
                          uint64_t c1, bool clear_status, uint32_t warps_per_block) {
  const uint32_t S = p->symbol_bytes, C = p->chunk_bytes;
  const uint64_t nc = div_up(n_bytes, C);
  if (c1 > nc) c1 = nc;
  if (c0 >= c1 && nc > 0) return LZ_OK;
  const uint64_t records_at = glz::kHeaderBytes + glz::kTableEntry * nc +
                              8ull * div_up(nc, glz::kIndexStride);
  const uint32_t offB = off_bytes(p->window);
  if (nc == 0)
    return cuda_status(glz::launch_header(static_cast<uint8_t *>(d_out), version, S, offB,
                                          p->min_match, p->max_match, C,
                                          p->window, out_bytes, st));

  glz::CompressSmem sm = compress_layout(p);
  if (static_cast<int64_t>(sm.per_warp) > ctx->smem_optin) return LZ_ERR_INVALID_ARG;
  int block = 32;
  int64_t best_blocks = 1;
  if (!block_shape(sm.per_warp, ctx->smem_per_sm, ctx->smem_reserved, ctx->smem_optin,
                   warps_per_block, &block, &best_blocks))
    return LZ_ERR_INVALID_ARG;
  const uint64_t wpb = block / 32;
  uint64_t grid = div_up(c1 - c0, wpb);
  if (grid > static_cast<uint64_t>(best_blocks) * ctx->sms) grid = best_blocks * ctx->sms;
  // scratch: work counter, nc status words, parking slots of every warp
  const uint32_t slot_bytes =
      round16(record_bound(C / S, S, off_bytes(p->window), p->min_match) + S + 16);
  const size_t status_end = kScratchHead + 8ull * nc;
  const size_t park_at = (status_end + 255) & ~static_cast<size_t>(255);
  // a launch over part of the chunks (one piece of lz_compress_host) keeps
  // the status words of the launches before it, so the scratch must not be
  // reallocated between them: it is sized for the largest grid
  const uint64_t grid_room =
      (c0 > 0 || c1 < nc) ? static_cast<uint64_t>(best_blocks) * ctx->sms : grid;
  const size_t need = park_at + static_cast<size_t>(slot_bytes) * kParkSlots * wpb * grid_room;
  lz_status s = reserve_scratch(ctx, need);
  if (s != LZ_OK) return s;
  cudaError_t e = cudaMemsetAsync(ctx->scratch, 0, clear_status ? status_end : kScratchHead, st);
  if (e != cudaSuccess) return LZ_ERR_CUDA;

  glz::CompressArgs A{};
  A.buf.in = static_cast<const uint8_t *>(d_in);
  A.buf.n = n_bytes;
  A.buf.out = static_cast<uint8_t *>(d_out);
  A.buf.cap = out_cap;
  A.buf.out_bytes = out_bytes;
  A.buf.S = S;
  A.buf.C = C;
  A.buf.W = p->window;
  A.buf.m = p->min_match;
  A.buf.M = p->max_match;
  A.buf.offB = offB;
  A.buf.nc = static_cast<uint32_t>(nc);
  A.buf.records_at = records_at;
  A.buf.in_aligned = (reinterpret_cast<uintptr_t>(d_in) % 16) == 0;
  A.buf.match = match == LZ_MATCH_PAPER     ? glz::kMatchPaper
                : match == LZ_MATCH_OVERLAP ? glz::kMatchOverlap
                                            : glz::kMatchExact;
  A.buf.version = version;
  A.buf.gbase = 0;
  A.total_chunks = nc;
  A.sm = sm;
  A.park = static_cast<uint8_t *>(ctx->scratch) + park_at;
  A.park_slots = kParkSlots;
  A.park_slot_bytes = slot_bytes;
  A.ticket = static_cast<uint32_t *>(ctx->scratch);
  A.status = reinterpret_cast<unsigned long long *>(
      static_cast<uint8_t *>(ctx->scratch) + kScratchHead);
  A.err = ctx->d_err;
  A.spin_limit = ctx->hooks.spin_limit ? ctx->hooks.spin_limit : glz::kSpinLimit;
  A.first_ticket = static_cast<uint32_t>(c0 + ctx->hooks.first_chunk);
  A.end_chunk = static_cast<uint32_t>(c1);
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

// Piece sizes for lz_compress_host: whole multiples of `sb` except the last
// (which takes the rest), growing from 8 MiB to 64 MiB at the start and
// shrinking back to 8 MiB at the end.
std::vector<uint64_t> host_pieces(uint64_t n, uint64_t sb) {
  const auto whole = [&](uint64_t v) { return std::max<uint64_t>(sb, (v / sb) * sb); };
  const uint64_t small = whole(8ull << 20), big = whole(64ull << 20);
  std::vector<uint64_t> tail, out;
  uint64_t left = (n / sb) * sb;  // the ragged rest joins the last piece
  for (uint64_t s = small; left > 0 && s < big; s *= 2) {  // the end, last first
    const uint64_t t = std::min(left, whole(s));
    tail.push_back(t);
    left -= t;
  }
  for (uint64_t s = small; left > 0 && s < big; s *= 2) {  // the start
    const uint64_t t = std::min(left, whole(s));
    out.push_back(t);
    left -= t;
  }
  while (left > 0) {
    const uint64_t t = std::min(left, big);
    out.push_back(t);
    left -= t;
  }
  out.insert(out.end(), tail.rbegin(), tail.rend());
  if (out.empty()) out.push_back(0);
  out.back() += n - (n / sb) * sb;
  return out;
}

}  // namespace

extern "C" {

lz_status lz_compress_host(lz_ctx *ctx, const void *h_in, uint64_t n_bytes, const lz_params *p,
                           void *h_out, uint64_t out_cap, uint64_t *h_out_bytes,
                           lz_stream_t stream) {
  if (!ctx || !params_ok(p) || !h_out || !h_out_bytes || (n_bytes > 0 && !h_in))
    return LZ_ERR_INVALID_ARG;
  const uint32_t S = p->symbol_bytes, C = p->chunk_bytes;
  if (n_bytes % S != 0) return LZ_ERR_INVALID_ARG;
  const uint64_t nc = div_up(n_bytes, C);
  if (nc > kMaxLaunchChunks) return LZ_ERR_INVALID_ARG;
  const uint64_t records_at = glz::kHeaderBytes + glz::kTableEntry * nc +
                              8ull * div_up(nc, glz::kIndexStride);
  if (out_cap < records_at) return LZ_ERR_BUFFER_TOO_SMALL;
  std::lock_guard<std::mutex> lock(ctx->mu);
  if (cudaSetDevice(ctx->device) != cudaSuccess) return LZ_ERR_CUDA;
  cudaError_t e = cudaSuccess;
  for (int i = 0; i < 3 && e == cudaSuccess; ++i)
    if (!ctx->hs[i]) e = cudaStreamCreateWithFlags(&ctx->hs[i], cudaStreamNonBlocking);
  for (int i = 0; i < 17 && e == cudaSuccess; ++i)
    if (!ctx->hev[i]) e = cudaEventCreateWithFlags(&ctx->hev[i], cudaEventDisableTiming);
  if (e == cudaSuccess && !ctx->hpin)
    e = cudaHostAlloc(reinterpret_cast<void **>(&ctx->hpin), 8 * sizeof(uint64_t),
                      cudaHostAllocDefault);
  if (e != cudaSuccess) return cuda_status(e);
  // The stream is built in device memory.  A pinned h_out gets it piece by
  // piece: once a piece's launch is done, the look-back word of its last
  // chunk gives the end of the records written so far, and a copy on a
  // third stream takes them to h_out while later pieces are copied in and
  // compressed (copy engines in both directions: the host link carries
  // both at once).  A pageable h_out gets one copy at the end.
  bool pinned = false;
  {
    cudaPointerAttributes at{};
    pinned = cudaPointerGetAttributes(&at, h_out) == cudaSuccess &&
             at.type == cudaMemoryTypeHost;
    cudaGetLastError();  // clear a lookup error of an unregistered pointer
  }
  const uint64_t in_room = (n_bytes + 255) & ~255ull;
  const uint64_t cap = std::min(out_cap, lz_compressed_bound(n_bytes, p));
  const uint64_t out_room = (cap + 255) & ~255ull;
  const uint64_t want = in_room + 256 + out_room;
  if (ctx->hdev_bytes < want) {
    if (ctx->hooks.fail_alloc) return LZ_ERR_NOMEM;
    if (ctx->hdev) cudaFree(ctx->hdev);
    ctx->hdev = nullptr;
    ctx->hdev_bytes = 0;
    if ((e = cudaMalloc(&ctx->hdev, want)) != cudaSuccess) return cuda_status(e);
    ctx->hdev_bytes = want;
  }
  uint8_t *d_in = static_cast<uint8_t *>(ctx->hdev);
  auto *d_size = reinterpret_cast<unsigned long long *>(d_in + in_room);
  uint8_t *d_out = d_in + in_room + 256;
  uint8_t *hb = static_cast<uint8_t *>(h_out);
  cudaStream_t s_in = ctx->hs[0], s_comp = ctx->hs[1], s_out = ctx->hs[2];
  cudaEvent_t ev_start = ctx->hev[16];
  if (cudaEventRecord(ev_start, reinterpret_cast<cudaStream_t>(stream)) != cudaSuccess ||
      cudaStreamWaitEvent(s_in, ev_start, 0) != cudaSuccess ||
      cudaStreamWaitEvent(s_comp, ev_start, 0) != cudaSuccess ||
      cudaStreamWaitEvent(s_out, ev_start, 0) != cudaSuccess)
    return LZ_ERR_CUDA;
  // records [records_at, copied) are on their way to h_out
  uint64_t copied = records_at;
  bool copying = pinned;
  // piece j is done: copy the records it completed (from a 64-byte boundary:
  // the bytes before are final or rewritten by the copy of the table at the
  // end)
  auto flush = [&](size_t j) {
    if (!copying) return;
    cudaEvent_t done = ctx->hev[8 + j % 8];
    if (cudaEventSynchronize(done) != cudaSuccess) {
      copying = false;
      return;
    }
    const uint64_t w = ctx->hpin[j % 8];
    if (!(w & kStatusPrefix)) {  // not placed: a device error, reported below
      copying = false;
      return;
    }
    const uint64_t end = std::min(cap, records_at + (w & kStatusValue));
    if (end <= copied) return;
    const uint64_t from = copied & ~63ull;
    if (cudaStreamWaitEvent(s_out, done, 0) != cudaSuccess ||
        cudaMemcpyAsync(hb + from, d_out + from, end - from, cudaMemcpyDeviceToHost, s_out) !=
            cudaSuccess) {
      copying = false;
      return;
    }
    copied = end;
  };
  lz_status st = LZ_OK;
  if (nc == 0) {
    st = compress_locked(ctx, d_in, 0, p, LZ_MATCH_EXACT, 1, d_out, cap, d_size, s_comp);
  } else {
    // pieces of whole index superblocks: the copy of piece i + 1 overlaps
    // the compression of piece i; a launch takes only its piece's chunks,
    // and its look-back reaches into the pieces before it.  Pieces of about
    // 64 MiB in the middle (4 MiB pieces throughout measured 26 % slower end
    // to end, 16 MiB 3 %: each piece costs a launch and an event wait), but
    // small at both ends, where nothing overlaps: compression starts once
    // the first piece is in, and the call ends once the last one is out
    const uint64_t sb = glz::kIndexStride * static_cast<uint64_t>(C);
    const std::vector<uint64_t> pieces = host_pieces(n_bytes, sb);
    uint64_t at = 0;
    for (size_t i = 0; i < pieces.size() && st == LZ_OK; ++i) {
      const uint64_t len = pieces[i];
      const uint64_t c0 = at / C, c1 = (at + len) / C + ((at + len) % C ? 1 : 0);
      cudaEvent_t ev = ctx->hev[i % 8];
      if (cudaMemcpyAsync(d_in + at, static_cast<const uint8_t *>(h_in) + at, len,
                          cudaMemcpyHostToDevice, s_in) != cudaSuccess ||
          cudaEventRecord(ev, s_in) != cudaSuccess ||
          cudaStreamWaitEvent(s_comp, ev, 0) != cudaSuccess) {
        st = LZ_ERR_CUDA;
        break;
      }
      st = compress_locked(ctx, d_in, n_bytes, p, LZ_MATCH_EXACT, 1, d_out, cap, d_size, s_comp,
                           c0, c1, i == 0);
      at += len;
      if (st != LZ_OK || !pinned) continue;
      // the look-back word of the piece's last chunk (its records' end)
      const auto *word = reinterpret_cast<const uint64_t *>(
          static_cast<const uint8_t *>(ctx->scratch) + kScratchHead + 8 * (c1 - 1));
      if (cudaMemcpyAsync(&ctx->hpin[i % 8], word, 8, cudaMemcpyDeviceToHost, s_comp) !=
              cudaSuccess ||
          cudaEventRecord(ctx->hev[8 + i % 8], s_comp) != cudaSuccess) {
        st = LZ_ERR_CUDA;
        break;
      }
      // the host waits for the oldest piece whose records are not on their
      // way yet, while the GPU has the next pieces queued
      if (i >= kHostLag) flush(i - kHostLag);
    }
    for (size_t j = pieces.size() > kHostLag ? pieces.size() - kHostLag : 0;
         st == LZ_OK && pinned && j < pieces.size(); ++j)
      flush(j);
  }
  uint64_t size = 0;
  if (st == LZ_OK &&
      (cudaMemcpyAsync(&size, d_size, 8, cudaMemcpyDeviceToHost, s_comp) != cudaSuccess ||
       cudaStreamSynchronize(s_comp) != cudaSuccess))
    st = LZ_ERR_CUDA;
  cudaStreamSynchronize(s_in);
  cudaStreamSynchronize(s_comp);
  // device-side errors of this call, returned here (and cleared)
  uint32_t h = 0;
  if (cudaMemcpyAsync(&h, ctx->d_err, 4, cudaMemcpyDeviceToHost, s_comp) != cudaSuccess ||
      cudaStreamSynchronize(s_comp) != cudaSuccess) {
    if (st == LZ_OK) st = LZ_ERR_CUDA;
  }
  if (h) {
    cudaMemsetAsync(ctx->d_err, 0, 4, s_comp);
    cudaStreamSynchronize(s_comp);
    if (st == LZ_OK && !(h == glz::kErrSmall))
      st = (h & glz::kErrInternal)  ? LZ_ERR_INTERNAL
           : (h & glz::kErrTimeout) ? LZ_ERR_TIMEOUT
           : (h & glz::kErrCorrupt) ? LZ_ERR_CORRUPT
                                    : LZ_ERR_BUFFER_TOO_SMALL;
  }
  if (st != LZ_OK) {
    cudaStreamSynchronize(s_out);
    return st;
  }
  *h_out_bytes = size;
  if (size > out_cap) {
    cudaStreamSynchronize(s_out);
    return LZ_ERR_BUFFER_TOO_SMALL;
  }
  // the header, table and index (final now), and any records not yet copied
  const uint64_t head = std::min<uint64_t>(records_at, size);
  bool ok = cudaMemcpyAsync(hb, d_out, head, cudaMemcpyDeviceToHost, s_out) == cudaSuccess;
  if (ok && size > copied && pinned)
    ok = cudaMemcpyAsync(hb + copied, d_out + copied, size - copied, cudaMemcpyDeviceToHost,
                         s_out) == cudaSuccess;
  if (ok && !pinned && size > head)
    ok = cudaMemcpyAsync(hb + head, d_out + head, size - head, cudaMemcpyDeviceToHost, s_out) ==
         cudaSuccess;
  if (cudaStreamSynchronize(s_out) != cudaSuccess || !ok) return LZ_ERR_CUDA;
  return LZ_OK;
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
  if (std::memcmp(h, "GLZ1", 4) != 0 || (h[4] != 1 && h[4] != 2) || h[9] > (h[4] == 2 ? 1 : 0) || h[10] || h[11] ||
      !params_ok(&p) || h[6] != off_bytes(p.window) || (h[4] == 1 && n % p.symbol_bytes != 0) ||
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
  A.smem_bytes = decode_block_smem(ctx);
  return cuda_status(glz::launch_decompress(A, kDecompressBlock,
                                            reinterpret_cast<cudaStream_t>(stream)));
}

lz_status lz_stitch(lz_ctx *ctx, const void *d_shard, uint64_t shard_bytes,
                    uint64_t shard_chunks, uint64_t chunk_base, uint64_t total_chunks,
                    uint64_t total_bytes, uint64_t record_base, void *d_out,
                    uint64_t out_cap, lz_stream_t stream) {
  if (!ctx || !d_shard || !d_out) return LZ_ERR_INVALID_ARG;
  if (reinterpret_cast<uintptr_t>(d_shard) % 8 != 0 ||
      reinterpret_cast<uintptr_t>(d_out) % 8 != 0)
    return LZ_ERR_INVALID_ARG;
  if (total_chunks > 0xFFFFFFFFull || shard_chunks > total_chunks ||
      chunk_base > total_chunks - shard_chunks)
    return LZ_ERR_INVALID_ARG;
  if (shard_chunks > 0 && chunk_base % glz::kIndexStride != 0) return LZ_ERR_INVALID_ARG;
  const uint64_t src_records = glz::kHeaderBytes + glz::kTableEntry * shard_chunks +
                               8ull * div_up(shard_chunks, glz::kIndexStride);
  if (shard_bytes < src_records) return LZ_ERR_INVALID_ARG;
  const uint64_t records_at = glz::kHeaderBytes + glz::kTableEntry * total_chunks +
                              8ull * div_up(total_chunks, glz::kIndexStride);
  const uint64_t record_bytes = shard_bytes - src_records;
  if (out_cap < records_at || record_base > out_cap - records_at ||
      record_bytes > out_cap - records_at - record_base)
    return LZ_ERR_BUFFER_TOO_SMALL;
  glz::StitchArgs A{};
  A.shard = static_cast<const uint8_t *>(d_shard);
  A.shard_chunks = shard_chunks;
  A.chunk_base = chunk_base;
  A.total_chunks = total_chunks;
  A.total_bytes = total_bytes;
  A.record_base = record_base;
  A.src_records = src_records;
  A.record_bytes = record_bytes;
  A.dst_records = records_at + record_base;
  A.out = static_cast<uint8_t *>(d_out);
  A.err = ctx->d_err;
  std::lock_guard<std::mutex> lock(ctx->mu);
  if (cudaSetDevice(ctx->device) != cudaSuccess) return LZ_ERR_CUDA;
  return cuda_status(
      glz::launch_stitch(A, ctx->sms, reinterpret_cast<cudaStream_t>(stream)));
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
    return cuda_status(glz::launch_header(static_cast<uint8_t *>(d_out), 1u, S, offB,
                                          p->min_match, p->max_match, C, p->window,
                                          out_bytes, st));
  const glz::CompressSmem sm = compress_layout(p);
  if (static_cast<int64_t>(sm.per_warp) > nd->smem_optin) return LZ_ERR_INVALID_ARG;
  int block = 32;
  int64_t best_blocks = 1;
  if (!block_shape(sm.per_warp, nd->smem_per_sm, nd->smem_reserved, nd->smem_optin, 0, &block,
                   &best_blocks))
    return LZ_ERR_INVALID_ARG;
  uint64_t grid = div_up(nc, block / 32);
  if (grid > static_cast<uint64_t>(best_blocks) * nd->sms) grid = best_blocks * nd->sms;
  // the counter, the error word and the status words start at zero (one
  // clear, so that an error left by an earlier failed call cannot leak in)
  if (cudaMemsetAsync(nd->scratch, 0, kNoAllocHead + 8ull * nc, st) != cudaSuccess)
    return LZ_ERR_CUDA;
  glz::CompressArgs A{};
  A.buf.in = static_cast<const uint8_t *>(d_in);
  A.buf.n = n_bytes;
  A.buf.out = static_cast<uint8_t *>(d_out);
  A.buf.cap = out_cap;
  A.buf.out_bytes = out_bytes;
  A.buf.S = S;
  A.buf.C = C;
  A.buf.W = p->window;
  A.buf.m = p->min_match;
  A.buf.M = p->max_match;
  A.buf.offB = offB;
  A.buf.nc = static_cast<uint32_t>(nc);
  A.buf.records_at = records_at;
  A.buf.in_aligned = (reinterpret_cast<uintptr_t>(d_in) % 16) == 0;
  A.buf.gbase = 0;
  A.total_chunks = nc;
  A.sm = sm;
  A.park = nullptr;  // no parking slots: blocking look-back
  A.park_slots = 0;
  A.park_slot_bytes = 0;
  A.ticket = reinterpret_cast<uint32_t *>(nd->scratch);
  A.err = reinterpret_cast<uint32_t *>(nd->scratch + 4);
  A.spin_limit = glz::kSpinLimit;
  A.end_chunk = static_cast<uint32_t>(nc);
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

// ---------------------------------------------------------------------------
// Batches: many buffers in one persistent launch.

// Device buffers a batch owns, one slot each; a re-plan (lz_batch_update)
// reuses a slot when it is large enough.
enum BatchBuf { kBufScratch, kBufItems, kBufBases, kBufEmpties, kBufIns, kBufInBytes, kBufHdr,
                kBufCount };

struct DevBuf {
  void *p = nullptr;
  size_t cap = 0;
};

struct lz_batch {
  int decompress = 0;
  int device = 0;
  int planned = 0;                // 1 once a plan succeeded (runs allowed)
  int fail_alloc = 0;             // the context's injected allocation failure (test hook)
  uint32_t match = 0, version = 1;  // compression options of every plan
  uint32_t warps_per_block = 0;
  cudaStream_t stream = nullptr;  // allocations and uploads are ordered on it
  DevBuf bufs[kBufCount];         // device allocations owned by the batch
  // compression
  glz::CompressArgs cargs{};
  const glz::BufDesc *d_empty = nullptr;
  uint32_t n_empty = 0, nj = 1;
  int block = 32;
  unsigned grid = 1;
  size_t clear_bytes = 0;
  void *scratch = nullptr;
  // decompression
  glz::DecompressBatchArgs dargs{};
  int dblock = 256;
};

namespace {

// Device memory for slot `slot` of at least `bytes`, stream-ordered on the
// batch's stream (no device-wide sync): the slot's buffer when it is large
// enough, else a new one (the old one is freed after the work already
// enqueued on that stream).  A new buffer has room for half as much again,
// so that a batch re-planned with a few more items keeps its memory.
lz_status batch_alloc(lz_batch *b, int slot, size_t bytes, void **p) {
  *p = nullptr;
  if (bytes == 0) return LZ_OK;
  DevBuf &d = b->bufs[slot];
  if (d.cap < bytes) {
    if (b->fail_alloc) return LZ_ERR_NOMEM;  // injected failure (test hook)
    if (d.p) cudaFreeAsync(d.p, b->stream);
    d.p = nullptr;
    d.cap = 0;
    const size_t want = bytes + bytes / 2;
    cudaError_t e = cudaMallocAsync(&d.p, want, b->stream);
    if (e != cudaSuccess) return cuda_status(e);
    d.cap = want;
  }
  *p = d.p;
  return LZ_OK;
}

// Upload a host array into slot `slot` (pageable: the call returns once the
// data is staged).
template <typename T>
lz_status batch_upload(lz_batch *b, int slot, const std::vector<T> &v, const T **dst) {
  void *p = nullptr;
  lz_status s = batch_alloc(b, slot, v.size() * sizeof(T), &p);
  if (s != LZ_OK) return s;
  if (!v.empty() && cudaMemcpyAsync(p, v.data(), v.size() * sizeof(T),
                                    cudaMemcpyHostToDevice, b->stream) != cudaSuccess)
    return LZ_ERR_CUDA;
  *dst = static_cast<const T *>(p);
  return LZ_OK;
}

// Per-warp slice covering every parameter set of a batch: each region at its
// largest size.
glz::CompressSmem compress_layout_max(const std::vector<lz_params> &ps) {
  uint64_t in = 16, links = 16, flags = 16, pay = 16, maybe = 16;
  for (const lz_params &p : ps) {
    const glz::CompressSmem one = compress_layout(&p);
    in = std::max<uint64_t>(in, one.prev_off - one.in_off);
    links = std::max<uint64_t>(links, one.flags_off - one.prev_off);
    flags = std::max<uint64_t>(flags, one.pay_off - one.flags_off);
    pay = std::max<uint64_t>(pay, one.pay_bytes);
    maybe = std::max<uint64_t>(maybe, one.mbar_off - one.maybe_off);
  }
  glz::CompressSmem sm{};
  uint32_t at = 0;
  sm.in_off = at;
  at += static_cast<uint32_t>(in);
  sm.prev_off = at;
  at += static_cast<uint32_t>(links);
  sm.flags_off = at;
  at += static_cast<uint32_t>(flags);
  sm.pay_off = at;
  sm.pay_bytes = static_cast<uint32_t>(pay);
  at += static_cast<uint32_t>(pay);
  sm.maybe_off = at;
  at += static_cast<uint32_t>(maybe);
  sm.mbar_off = at;
  at += 16;
  sm.per_warp = (at + 127) & ~127u;
  uint32_t lg = 1;
  while (lg < 15 && (2u << (lg + 1)) <= sm.pay_bytes) ++lg;
  sm.hash_log2 = lg;
  return sm;
}

lz_status batch_create_compress(lz_ctx *ctx, const lz_batch_item *items, uint32_t n,
                                lz_batch *b, uint32_t match, uint32_t version) {
  const uint32_t warps_per_block = b->warps_per_block;
  std::vector<glz::BufDesc> descs, empties;
  std::vector<uint64_t> bases;
  std::vector<lz_params> ps;
  uint64_t total = 0, kmax = 1;
  uint32_t nj = 1;
  for (uint32_t i = 0; i < n; ++i) {
    const lz_batch_item &it = items[i];
    const lz_params *p = &it.params;
    if (!params_ok(p) || !it.d_out || !it.d_out_bytes) return LZ_ERR_INVALID_ARG;
    if (reinterpret_cast<uintptr_t>(it.d_out_bytes) % 8 != 0) return LZ_ERR_INVALID_ARG;
    if (it.in_bytes > 0 && !it.d_in) return LZ_ERR_INVALID_ARG;
    if (version == 1 && it.in_bytes % p->symbol_bytes != 0) return LZ_ERR_INVALID_ARG;
    const uint64_t nc = div_up(it.in_bytes, p->chunk_bytes);
    if (nc > 0xFFFFFFFFull) return LZ_ERR_INVALID_ARG;
    const uint64_t records_at = glz::kHeaderBytes + glz::kTableEntry * nc +
                                8ull * div_up(nc, glz::kIndexStride);
    if (it.out_cap < records_at) return LZ_ERR_BUFFER_TOO_SMALL;
    glz::BufDesc d{};
    d.in = static_cast<const uint8_t *>(it.d_in);
    d.n = it.in_bytes;
    d.out = static_cast<uint8_t *>(it.d_out);
    d.cap = it.out_cap;
    d.out_bytes = reinterpret_cast<unsigned long long *>(it.d_out_bytes);
    d.S = p->symbol_bytes;
    d.C = p->chunk_bytes;
    d.W = p->window;
    d.m = p->min_match;
    d.M = p->max_match;
    d.offB = off_bytes(p->window);
    d.nc = static_cast<uint32_t>(nc);
    d.in_aligned = (reinterpret_cast<uintptr_t>(it.d_in) % 16) == 0;
    d.records_at = records_at;
    d.gbase = total;
    d.match = match;
    d.version = version;
    if (nc == 0) {
      empties.push_back(d);
      continue;
    }
    descs.push_back(d);
    bases.push_back(total);
    total += nc;
    if (total > kMaxLaunchChunks) return LZ_ERR_INVALID_ARG;
    ps.push_back(*p);
    kmax = std::max<uint64_t>(kmax, p->chunk_bytes / p->symbol_bytes);
    uint32_t j = 1;
    while (32 * j < p->window) j *= 2;
    nj = std::max(nj, j);
  }
  glz::CompressSmem sm = ps.empty() ? glz::CompressSmem{} : compress_layout_max(ps);
  if (!ps.empty() && static_cast<int64_t>(sm.per_warp) > ctx->smem_optin)
    return LZ_ERR_INVALID_ARG;
  int block = 32;
  int64_t best_blocks = 1;
  if (!ps.empty() && !block_shape(sm.per_warp, ctx->smem_per_sm, ctx->smem_reserved,
                                  ctx->smem_optin, warps_per_block, &block, &best_blocks))
    return LZ_ERR_INVALID_ARG;
  const uint64_t wpb = block / 32;
  uint64_t grid = std::max<uint64_t>(1, div_up(total, wpb));
  if (grid > static_cast<uint64_t>(best_blocks) * ctx->sms) grid = best_blocks * ctx->sms;
  uint64_t rb_max = 0;  // a parking slot holds any item's largest record
  for (const lz_params &q : ps)
    rb_max = std::max<uint64_t>(rb_max, record_bound(q.chunk_bytes / q.symbol_bytes,
                                                     q.symbol_bytes, off_bytes(q.window),
                                                     q.min_match) +
                                            q.symbol_bytes);
  const uint32_t slot_bytes = round16(rb_max + 16);
  const size_t status_end = kScratchHead + 8ull * total;
  const size_t park_at = (status_end + 255) & ~static_cast<size_t>(255);
  const size_t scratch = park_at + static_cast<size_t>(slot_bytes) * kParkSlots * wpb * grid;
  lz_status s = batch_alloc(b, kBufScratch, scratch, &b->scratch);
  if (s != LZ_OK) return s;
  const glz::BufDesc *d_items = nullptr, *d_empty = nullptr;
  const uint64_t *d_base = nullptr;
  if ((s = batch_upload(b, kBufItems, descs, &d_items)) != LZ_OK) return s;
  if ((s = batch_upload(b, kBufBases, bases, &d_base)) != LZ_OK) return s;
  if ((s = batch_upload(b, kBufEmpties, empties, &d_empty)) != LZ_OK) return s;
  glz::CompressArgs &A = b->cargs;
  A.items = d_items;
  A.item_base = d_base;
  A.n_items = static_cast<uint32_t>(descs.size());
  A.total_chunks = total;
  A.sm = sm;
  A.ticket = static_cast<uint32_t *>(b->scratch);
  A.status = reinterpret_cast<unsigned long long *>(static_cast<uint8_t *>(b->scratch) +
                                                     kScratchHead);
  A.err = ctx->d_err;
  A.park = static_cast<uint8_t *>(b->scratch) + park_at;
  A.park_slots = kParkSlots;
  A.park_slot_bytes = slot_bytes;
  A.spin_limit = glz::kSpinLimit;
  A.first_ticket = 0;
  b->d_empty = d_empty;
  b->n_empty = static_cast<uint32_t>(empties.size());
  b->nj = nj;
  b->block = block;
  b->grid = static_cast<unsigned>(grid);
  b->clear_bytes = status_end;
  return LZ_OK;
}

uint64_t header_u(const uint8_t *h, int at, int n) {
  uint64_t v = 0;
  for (int i = 0; i < n; ++i) v |= static_cast<uint64_t>(h[at + i]) << (8 * i);
  return v;
}

lz_status batch_create_decompress(lz_ctx *ctx, const lz_batch_item *items, uint32_t n,
                                  lz_batch *b) {
  std::vector<const uint8_t *> ins(n);
  std::vector<uint64_t> in_bytes(n);
  for (uint32_t i = 0; i < n; ++i) {
    if (!items[i].d_in || !items[i].d_out_bytes) return LZ_ERR_INVALID_ARG;
    if (reinterpret_cast<uintptr_t>(items[i].d_out_bytes) % 8 != 0) return LZ_ERR_INVALID_ARG;
    if (items[i].in_bytes < glz::kHeaderBytes) return LZ_ERR_CORRUPT;
    ins[i] = static_cast<const uint8_t *>(items[i].d_in);
    in_bytes[i] = items[i].in_bytes;
  }
  // an item that states its stream's parameters (params.chunk_bytes != 0)
  // and, in out_cap, its exact decompressed size needs no header read; the
  // kernel still checks every header against the plan
  bool read = false;
  for (uint32_t i = 0; i < n; ++i) read = read || items[i].params.chunk_bytes == 0;
  std::vector<uint8_t> hdr(static_cast<size_t>(n) * 32);
  if (read) {
    const uint8_t *const *d_ins = nullptr;
    const uint64_t *d_inb = nullptr;
    lz_status s;
    if ((s = batch_upload(b, kBufIns, ins, &d_ins)) != LZ_OK) return s;
    if ((s = batch_upload(b, kBufInBytes, in_bytes, &d_inb)) != LZ_OK) return s;
    void *d_hdr = nullptr;
    if ((s = batch_alloc(b, kBufHdr, hdr.size(), &d_hdr)) != LZ_OK) return s;
    if (n) {
      glz::gather_headers<<<std::min<uint32_t>(1024, (n * 32 + 255) / 256), 256, 0,
                            b->stream>>>(d_ins, d_inb, n, static_cast<uint8_t *>(d_hdr));
      if (cudaMemcpyAsync(hdr.data(), d_hdr, hdr.size(), cudaMemcpyDeviceToHost,
                          b->stream) != cudaSuccess ||
          cudaStreamSynchronize(b->stream) != cudaSuccess)
        return LZ_ERR_CUDA;
    }
  }
  std::vector<glz::DecItem> descs, empties;
  std::vector<uint64_t> bases;
  uint64_t total = 0, max_rec = 0, max_k = 1, max_c = 16;
  bool need_hi = false, shared = true;
  for (uint32_t i = 0; i < n; ++i) {
    const uint8_t *h = &hdr[static_cast<size_t>(i) * 32];
    lz_params p;
    uint64_t nn, nc;
    if (items[i].params.chunk_bytes != 0) {
      p = items[i].params;
      if (!params_ok(&p)) return LZ_ERR_INVALID_ARG;
      nn = items[i].out_cap;
      nc = div_up(nn, p.chunk_bytes);
      if (nc > 0xFFFFFFFFull) return LZ_ERR_INVALID_ARG;
    } else {
      p = lz_params{h[5], static_cast<uint32_t>(header_u(h, 12, 4)),
                    static_cast<uint32_t>(header_u(h, 16, 4)), h[7], h[8]};
      nn = header_u(h, 24, 8);
      nc = header_u(h, 20, 4);
      if (std::memcmp(h, "GLZ1", 4) != 0 || (h[4] != 1 && h[4] != 2) ||
          h[9] > (h[4] == 2 ? 1 : 0) || h[10] || h[11] || !params_ok(&p) ||
          h[6] != off_bytes(p.window) || (h[4] == 1 && nn % p.symbol_bytes != 0) ||
          nc != div_up(nn, p.chunk_bytes))
        return LZ_ERR_CORRUPT;
    }
    if (items[i].out_cap < nn || (nn > 0 && !items[i].d_out)) return LZ_ERR_BUFFER_TOO_SMALL;
    glz::DecItem d{};
    d.in = ins[i];
    d.in_bytes = in_bytes[i];
    d.out = static_cast<uint8_t *>(items[i].d_out);
    d.out_cap = items[i].out_cap;
    d.out_bytes = reinterpret_cast<unsigned long long *>(items[i].d_out_bytes);
    d.nc = static_cast<uint32_t>(nc);
    d.out_aligned = (reinterpret_cast<uintptr_t>(items[i].d_out) % 16) == 0;
    d.gbase = total;
    if (nc == 0) {
      empties.push_back(d);
      continue;
    }
    descs.push_back(d);
    bases.push_back(total);
    total += nc;
    const uint64_t k = p.chunk_bytes / p.symbol_bytes;
    max_k = std::max(max_k, k);
    max_c = std::max<uint64_t>(max_c, p.chunk_bytes);
    need_hi = need_hi || (p.symbol_bytes == 1 && off_bytes(p.window) == 2);
    shared = shared && p.symbol_bytes * p.min_match >= 1 + off_bytes(p.window);
    max_rec = std::max(max_rec, glz::decode_record_bound(k, p.symbol_bytes,
                                                         off_bytes(p.window), p.min_match));
  }
  const uint32_t budget = decode_block_smem(ctx);
  const glz::DecodeLayout lay =
      glz::decode_layout(max_k, max_c, max_rec, need_hi, shared, budget);
  if (lay.per_warp > budget) return LZ_ERR_INVALID_ARG;
  const uint64_t warps = std::min<uint64_t>(32, budget / lay.per_warp);
  const glz::DecItem *d_items = nullptr, *d_empty = nullptr;
  const uint64_t *d_base = nullptr;
  lz_status s;
  if ((s = batch_upload(b, kBufItems, descs, &d_items)) != LZ_OK) return s;
  if ((s = batch_upload(b, kBufBases, bases, &d_base)) != LZ_OK) return s;
  if ((s = batch_upload(b, kBufEmpties, empties, &d_empty)) != LZ_OK) return s;
  glz::DecompressBatchArgs &B = b->dargs;
  B.items = d_items;
  B.item_base = d_base;
  B.n_items = static_cast<uint32_t>(descs.size());
  B.total_chunks = total;
  B.empties = d_empty;
  B.n_empty = static_cast<uint32_t>(empties.size());
  B.lay = lay;
  B.smem_bytes = static_cast<uint32_t>(lay.per_warp * warps);
  B.err = ctx->d_err;
  b->dblock = static_cast<int>(32 * warps);
  return LZ_OK;
}

}  // namespace

extern "C" {

lz_status lz_batch_create(lz_ctx *ctx, const lz_batch_item *items, uint32_t n_items,
                          int decompress, lz_stream_t stream, lz_batch **out) {
  return lz_batch_create_ex(ctx, items, n_items, decompress, nullptr, stream, out);
}

lz_status lz_batch_create_ex(lz_ctx *ctx, const lz_batch_item *items, uint32_t n_items,
                             int decompress, const lz_options *opt, lz_stream_t stream,
                             lz_batch **out) {
  if (!ctx || !out || (n_items > 0 && !items)) return LZ_ERR_INVALID_ARG;
  const uint32_t match = opt ? opt->match : LZ_MATCH_EXACT;
  const uint32_t version = opt && opt->version ? opt->version : 1u;
  if (match != LZ_MATCH_EXACT && match != LZ_MATCH_PAPER && match != LZ_MATCH_OVERLAP)
    return LZ_ERR_INVALID_ARG;
  if ((version != 1 && version != 2) || (match == LZ_MATCH_OVERLAP && version != 2))
    return LZ_ERR_INVALID_ARG;
  const uint32_t wpb = opt ? opt->warps_per_block : 0u;
  if (wpb && wpb != 1 && wpb != 2 && wpb != 4 && wpb != 8) return LZ_ERR_INVALID_ARG;
  *out = nullptr;
  std::lock_guard<std::mutex> lock(ctx->mu);
  if (cudaSetDevice(ctx->device) != cudaSuccess) return LZ_ERR_CUDA;
  lz_batch *b = new (std::nothrow) lz_batch();
  if (!b) return LZ_ERR_NOMEM;
  b->fail_alloc = ctx->hooks.fail_alloc ? 1 : 0;
  b->decompress = decompress ? 1 : 0;
  b->device = ctx->device;
  b->stream = reinterpret_cast<cudaStream_t>(stream);
  b->match = match == LZ_MATCH_PAPER     ? glz::kMatchPaper
             : match == LZ_MATCH_OVERLAP ? glz::kMatchOverlap
                                         : glz::kMatchExact;
  b->version = version;
  b->warps_per_block = wpb;
  lz_status s = decompress ? batch_create_decompress(ctx, items, n_items, b)
                           : batch_create_compress(ctx, items, n_items, b, b->match, version);
  if (s != LZ_OK) {
    for (DevBuf &d : b->bufs)
      if (d.p) cudaFreeAsync(d.p, b->stream);
    delete b;
    return s;
  }
  b->planned = 1;
  *out = b;
  return LZ_OK;
}

lz_status lz_batch_update(lz_ctx *ctx, lz_batch *b, const lz_batch_item *items,
                          uint32_t n_items, lz_stream_t stream) {
  if (!ctx || !b || b->device != ctx->device || (n_items > 0 && !items))
    return LZ_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lock(ctx->mu);
  if (cudaSetDevice(ctx->device) != cudaSuccess) return LZ_ERR_CUDA;
  b->stream = reinterpret_cast<cudaStream_t>(stream);
  b->fail_alloc = ctx->hooks.fail_alloc ? 1 : 0;
  b->planned = 0;
  lz_status s = b->decompress ? batch_create_decompress(ctx, items, n_items, b)
                              : batch_create_compress(ctx, items, n_items, b, b->match,
                                                      b->version);
  if (s == LZ_OK) b->planned = 1;
  return s;
}

lz_status lz_batch_run(lz_ctx *ctx, lz_batch *b, lz_stream_t stream) {
  if (!ctx || !b || b->device != ctx->device || !b->planned) return LZ_ERR_INVALID_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (b->decompress) {
    if (b->dargs.total_chunks == 0 && b->dargs.n_empty == 0) return LZ_OK;
    b->dargs.err = ctx->d_err;
    return cuda_status(glz::launch_decompress_batch(b->dargs, b->dblock, st));
  }
  b->cargs.err = ctx->d_err;
  if (b->clear_bytes && cudaMemsetAsync(b->scratch, 0, b->clear_bytes, st) != cudaSuccess)
    return LZ_ERR_CUDA;
  return cuda_status(glz::launch_compress_batch(b->cargs, b->d_empty, b->n_empty, b->nj,
                                                b->block, b->grid, st));
}

void lz_batch_destroy(lz_batch *b, lz_stream_t stream) {
  if (!b) return;
  cudaSetDevice(b->device);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  for (DevBuf &d : b->bufs)
    if (d.p) cudaFreeAsync(d.p, st);
  delete b;
}

lz_status lz_autotune(lz_ctx *ctx, const void *d_sample, uint64_t sample_bytes,
                      uint32_t symbol_bytes, lz_params *out) {
  return lz_autotune_ex(ctx, d_sample, sample_bytes, symbol_bytes, out, nullptr, nullptr, 0,
                        nullptr);
}

lz_status lz_autotune_ex(lz_ctx *ctx, const void *d_sample, uint64_t sample_bytes,
                         uint32_t symbol_bytes, lz_params *out, uint32_t *out_warps_per_block,
                         lz_tune_trial *trials_out, uint32_t max_trials, uint32_t *n_trials) {
  if (!ctx || !d_sample || !out) return LZ_ERR_INVALID_ARG;
  if (symbol_bytes != 1 && symbol_bytes != 2 && symbol_bytes != 4) return LZ_ERR_INVALID_ARG;
  sample_bytes -= sample_bytes % symbol_bytes;
  if (sample_bytes == 0) return LZ_ERR_INVALID_ARG;
  const uint32_t Cs[4] = {2048, 4096, 8192, 16384};
  const uint32_t Ws[4] = {64, 128, 256, 512};
  const uint32_t m = symbol_bytes == 4 ? 2u : 3u;
  std::vector<lz_tune_trial> trials;
  uint64_t cap = 0;
  for (uint32_t C : Cs)
    for (uint32_t W : Ws) {
      lz_params p{symbol_bytes, C, W, m, 255};
      cap = std::max(cap, lz_compressed_bound(sample_bytes, &p));
      trials.push_back({p, 0, 0.0, 0.0});
    }
  if (cudaSetDevice(ctx->device) != cudaSuccess) return LZ_ERR_CUDA;
  void *d_out = nullptr, *d_nb = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  lz_status s = LZ_OK;
  if (ctx->hooks.fail_alloc || cudaMalloc(&d_out, cap) != cudaSuccess ||
      cudaMalloc(&d_nb, 8) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
      cudaEventCreate(&e1) != cudaSuccess)
    s = LZ_ERR_NOMEM;
  // one trial: three compressions (the first warms up), the mean of the
  // last two, and the ratio
  auto run = [&](lz_tune_trial &t) {
    lz_options opt{LZ_MATCH_EXACT, 1, t.warps_per_block};
    t.seconds = 0;
    for (int rep = 0; rep < 3 && s == LZ_OK; ++rep) {
      cudaEventRecord(e0, nullptr);
      s = lz_compress_ex(ctx, d_sample, sample_bytes, &t.params, &opt, d_out, cap,
                         static_cast<uint64_t *>(d_nb), nullptr);
      cudaEventRecord(e1, nullptr);
      if (s == LZ_OK) s = lz_sync(ctx, nullptr);
      float ms = 0;
      cudaEventElapsedTime(&ms, e0, e1);
      if (rep > 0) t.seconds += ms * 1e-3 / 2;
    }
    uint64_t size = 0;
    if (s == LZ_OK && cudaMemcpy(&size, d_nb, 8, cudaMemcpyDeviceToHost) != cudaSuccess)
      s = LZ_ERR_CUDA;
    t.ratio = size ? static_cast<double>(sample_bytes) / size : 0.0;
  };
  for (lz_tune_trial &t : trials) {
    if (s != LZ_OK) break;
    run(t);
  }
  lz_params best{};
  uint32_t best_wpb = 0;
  if (s == LZ_OK) {
    // among the sets whose ratio is within 5% of the best ratio seen, the
    // smallest chunk that is within 10% of the fastest time (a smaller chunk
    // needs less shared memory per warp, which matters when buffers of other
    // kinds share a batched launch), the fastest among those
    double best_ratio = 0;
    for (const lz_tune_trial &t : trials) best_ratio = std::max(best_ratio, t.ratio);
    double fastest = 0;
    for (const lz_tune_trial &t : trials)
      if (t.ratio >= 0.95 * best_ratio && (fastest == 0 || t.seconds < fastest))
        fastest = t.seconds;
    const lz_tune_trial *pick = nullptr;
    for (const lz_tune_trial &t : trials) {
      if (t.ratio < 0.95 * best_ratio || t.seconds > 1.1 * fastest) continue;
      if (!pick || t.params.chunk_bytes < pick->params.chunk_bytes ||
          (t.params.chunk_bytes == pick->params.chunk_bytes && t.seconds < pick->seconds))
        pick = &t;
    }
    best = pick->params;
    // then the launch shape for it: warps per block 1, 2, 4, 8 (the stream
    // is the same for all of them); the fastest, the library's own choice
    // (0) on a tie within 2%
    lz_tune_trial shape[5] = {{best, 0, 0, 0}, {best, 1, 0, 0}, {best, 2, 0, 0},
                              {best, 4, 0, 0}, {best, 8, 0, 0}};
    double fastest_shape = 0;
    for (lz_tune_trial &t : shape) {
      if (s != LZ_OK) break;
      if (t.warps_per_block &&
          static_cast<int64_t>(compress_layout(&best).per_warp) * t.warps_per_block >
              ctx->smem_optin)
        continue;  // this shape does not fit a block
      run(t);
      trials.push_back(t);
      if (t.warps_per_block == 0 || t.seconds < 0.98 * fastest_shape) {
        fastest_shape = t.seconds;
        best_wpb = t.warps_per_block;
      }
    }
  }
  if (s == LZ_OK) {
    *out = best;
    if (out_warps_per_block) *out_warps_per_block = best_wpb;
    if (trials_out)
      for (uint32_t i = 0; i < std::min<size_t>(max_trials, trials.size()); ++i)
        trials_out[i] = trials[i];
    if (n_trials) *n_trials = static_cast<uint32_t>(trials.size());
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (d_out) cudaFree(d_out);
  if (d_nb) cudaFree(d_nb);
  return s;
}

// Parameter policy (section 3.2.3): multi-byte matching first, with the
// level's window enlarged S times; single-byte matching with the level's
// window when the sample's compression ratio is below 1.5.
static uint32_t min_profitable_match(uint32_t S, uint32_t W) {
  return (1u + off_bytes(W)) / S + 1u;
}

lz_status lz_select_params(lz_ctx *ctx, const void *d_sample, uint64_t sample_bytes,
                           uint32_t dtype_bytes, uint32_t level, uint32_t chunk_bytes,
                           lz_params *out, lz_stream_t stream) {
  static const uint32_t kLevelWindow[4] = {32, 64, 128, 255};
  if (!ctx || !out) return LZ_ERR_INVALID_ARG;
  if (dtype_bytes != 1 && dtype_bytes != 2 && dtype_bytes != 4) return LZ_ERR_INVALID_ARG;
  if (level < 1 || level > 4) return LZ_ERR_INVALID_ARG;
  const uint32_t Wl = kLevelWindow[level - 1];
  const lz_params single{1, chunk_bytes, Wl, min_profitable_match(1, Wl), 255};
  if (!params_ok(&single)) return LZ_ERR_INVALID_ARG;
  if (dtype_bytes == 1) {
    *out = single;
    return LZ_OK;
  }
  sample_bytes -= sample_bytes % dtype_bytes;
  if (sample_bytes == 0 || !d_sample) return LZ_ERR_INVALID_ARG;
  const uint32_t Wm = std::min<uint32_t>(glz::kMaxWindow, dtype_bytes * Wl);
  const lz_params multi{dtype_bytes, chunk_bytes, Wm, min_profitable_match(dtype_bytes, Wm), 255};
  const uint64_t cap = lz_compressed_bound(sample_bytes, &multi);
  if (cudaSetDevice(ctx->device) != cudaSuccess) return LZ_ERR_CUDA;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  void *d_out = nullptr, *d_nb = nullptr;
  lz_status s = LZ_OK;
  if (cudaMallocAsync(&d_out, cap, st) != cudaSuccess ||
      cudaMallocAsync(&d_nb, 8, st) != cudaSuccess)
    s = LZ_ERR_NOMEM;
  if (s == LZ_OK)
    s = lz_compress(ctx, d_sample, sample_bytes, &multi, d_out, cap,
                    static_cast<uint64_t *>(d_nb), stream);
  uint64_t size = 0;
  if (s == LZ_OK && cudaMemcpyAsync(&size, d_nb, 8, cudaMemcpyDeviceToHost, st) != cudaSuccess)
    s = LZ_ERR_CUDA;
  if (d_out) cudaFreeAsync(d_out, st);
  if (d_nb) cudaFreeAsync(d_nb, st);
  const lz_status sync = lz_sync(ctx, stream);
  if (s == LZ_OK) s = sync;
  if (s != LZ_OK) return s;
  // ratio n / size below 3/2, in integers
  *out = (2 * sample_bytes < 3 * size) ? single : multi;
  return LZ_OK;
}

// ---- Huffman stage (the paper's use case: Huffman coding after LZSS) ----------

uint64_t lz_huff_bound(uint64_t n_bytes) {
  const uint64_t nb = div_up(n_bytes, 32768);
  return glz::huff_layout_bits_at(n_bytes) + div_up(n_bytes * 12, 32) * 4 + 4 * nb;
}

lz_status lz_huff_compress(lz_ctx *ctx, const void *d_in, uint64_t n_bytes, void *d_out,
                           uint64_t out_cap, uint64_t *d_out_bytes, lz_stream_t stream) {
  if (!ctx || !d_out || !d_out_bytes) return LZ_ERR_INVALID_ARG;
  if (n_bytes > 0 && !d_in) return LZ_ERR_INVALID_ARG;
  if (reinterpret_cast<uintptr_t>(d_out) % 8 || reinterpret_cast<uintptr_t>(d_out_bytes) % 8)
    return LZ_ERR_INVALID_ARG;
  if (n_bytes > (1ull << 44)) return LZ_ERR_INVALID_ARG;
  if (out_cap < glz::huff_layout_bits_at(n_bytes)) return LZ_ERR_BUFFER_TOO_SMALL;
  std::lock_guard<std::mutex> lock(ctx->mu);
  if (cudaSetDevice(ctx->device) != cudaSuccess) return LZ_ERR_CUDA;
  lz_status s = reserve_scratch(ctx, 4096);
  if (s != LZ_OK) return s;
  auto *hist = static_cast<unsigned long long *>(ctx->scratch);
  auto *book = reinterpret_cast<uint32_t *>(static_cast<uint8_t *>(ctx->scratch) + 2048);
  return cuda_status(glz::launch_huff_compress(
      static_cast<const uint8_t *>(d_in), n_bytes, static_cast<uint8_t *>(d_out), out_cap,
      reinterpret_cast<unsigned long long *>(d_out_bytes), hist, book, ctx->d_err, ctx->sms,
      reinterpret_cast<cudaStream_t>(stream)));
}

lz_status lz_huff_decompressed_size(const void *d_in, uint64_t in_bytes, uint64_t *h_n,
                                    lz_stream_t stream) {
  if (!d_in || !h_n) return LZ_ERR_INVALID_ARG;
  if (in_bytes < 272) return LZ_ERR_CORRUPT;
  uint8_t h[16];
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (cudaMemcpyAsync(h, d_in, 16, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return LZ_ERR_CUDA;
  uint64_t n = 0;
  for (int i = 0; i < 8; ++i) n |= static_cast<uint64_t>(h[8 + i]) << (8 * i);
  const uint8_t blk[4] = {0x00, 0x80, 0x00, 0x00};  // 32768, little-endian
  if (std::memcmp(h, "GHF1", 4) != 0 || std::memcmp(h + 4, blk, 4) != 0 ||
      n > (1ull << 44) || glz::huff_layout_bits_at(n) > in_bytes)
    return LZ_ERR_CORRUPT;
  *h_n = n;
  return LZ_OK;
}

lz_status lz_huff_decompress(lz_ctx *ctx, const void *d_in, uint64_t in_bytes, void *d_out,
                             uint64_t out_cap, uint64_t *d_out_bytes, lz_stream_t stream) {
  if (!ctx || !d_in || !d_out_bytes) return LZ_ERR_INVALID_ARG;
  if (out_cap > 0 && !d_out) return LZ_ERR_INVALID_ARG;
  if (reinterpret_cast<uintptr_t>(d_in) % 8 || reinterpret_cast<uintptr_t>(d_out_bytes) % 8)
    return LZ_ERR_INVALID_ARG;
  if (in_bytes < 272) return LZ_ERR_CORRUPT;
  std::lock_guard<std::mutex> lock(ctx->mu);
  if (cudaSetDevice(ctx->device) != cudaSuccess) return LZ_ERR_CUDA;
  return cuda_status(glz::launch_huff_decompress(
      static_cast<const uint8_t *>(d_in), in_bytes, static_cast<uint8_t *>(d_out), out_cap,
      reinterpret_cast<unsigned long long *>(d_out_bytes), ctx->d_err, ctx->sms,
      reinterpret_cast<cudaStream_t>(stream)));
}

}  // extern "C"
