// decompress.cu -- the decompression kernel (one warp per chunk).
//
// The paper only reports decompression throughput (section 4.4) and gives
// no algorithm; this is the design used here.  The host knows nothing
// about the stream: every warp reads and checks the header itself, so the
// call needs no host synchronisation.  Per chunk:
//   * the record offset is the superblock index entry plus the record sizes
//     of the (at most 63) chunks before it in its superblock -- no scan
//     across the whole stream;
//   * tokens are decoded 32 at a time (lane = token): the flag bits give
//     each token's payload offset by popcount, a shuffle scan of token
//     lengths gives each token's output position;
//   * output positions are then produced 32 at a time (lane = position):
//     the owning token is found by a binary search over the 32 token start
//     positions (shuffles); a position inside a pointer copies from
//     position - offset, and chains whose source lies in the same 32
//     positions are resolved by pointer jumping (five shuffle rounds);
//     older sources are read from a ring of the last >= W+32 decoded
//     symbols in shared memory (offsets are at most W);
//   * the record (flags + payload) is first staged into the warp's shared
//     slice with a TMA bulk copy, so token decoding reads shared memory;
//   * symbols are stored straight to the output, 32*S contiguous bytes per
//     warp instruction.
#include <cuda_runtime.h>

#include <mutex>

#include "glz_common.h"
#include "glz_device.cuh"

namespace glz {

namespace {

struct Header {
  uint32_t version, overlap, S, offB, m, M, C, W, nc;
  uint64_t n;
};

__device__ __forceinline__ bool read_header(const uint8_t *in, Header &h) {
  const bool magic = in[0] == 'G' && in[1] == 'L' && in[2] == 'Z' &&
                     in[3] == '1' && (in[4] == 1 || in[4] == 2) &&
                     in[9] <= (in[4] == 2 ? 1 : 0) && in[10] == 0 && in[11] == 0;
  h.version = in[4];
  h.overlap = in[9];  // version 2: pointers may be longer than their offset
  h.S = in[5];
  h.offB = in[6];
  h.m = in[7];
  h.M = in[8];
  h.C = static_cast<uint32_t>(ld_le(in + 12, 4));
  h.W = static_cast<uint32_t>(ld_le(in + 16, 4));
  h.nc = static_cast<uint32_t>(ld_le(in + 20, 4));
  h.n = ld_le(in + 24, 8);
  bool ok = magic && (h.S == 1 || h.S == 2 || h.S == 4);
  ok = ok && h.C >= 16 && h.C <= kMaxChunk && h.C % 16 == 0;
  ok = ok && h.W >= 1 && h.W <= kMaxWindow;
  ok = ok && h.m >= 1 && h.m <= h.M && h.M <= 255;
  ok = ok && h.offB == (h.W <= 256 ? 1u : 2u);
  ok = ok && (h.version == 2 || h.n % h.S == 0);  // version 2 allows a tail
  ok = ok && static_cast<uint64_t>(h.nc) == (h.n + h.C - 1) / h.C;
  return ok;
}

__device__ __forceinline__ void store_symbol(uint8_t *dst, uint32_t v,
                                             uint32_t S, bool aligned) {
  if (aligned && S == 4) {
    *reinterpret_cast<uint32_t *>(dst) = v;
  } else if (aligned && S == 2) {
    *reinterpret_cast<uint16_t *>(dst) = static_cast<uint16_t>(v);
  } else {
    for (uint32_t i = 0; i < S; ++i) dst[i] = static_cast<uint8_t>(v >> (8 * i));
  }
}

// Sum of the record sizes of chunks [lo, hi) (hi - lo <= 64).
__device__ __forceinline__ uint64_t record_bytes(const uint8_t *table,
                                                 uint32_t lo, uint32_t hi,
                                                 uint32_t lane) {
  uint64_t part = 0;
  for (uint32_t e = lo + lane; e < hi; e += 32) {
    const uint64_t ntok = ld_le(table + 8ull * e, 4);
    const uint64_t pay = ld_le(table + 8ull * e + 4, 4);
    part += (ntok + 7) / 8 + pay;
  }
  return warp_sum_u64(part);
}

// Worst-case record of a chunk of k symbols (flags + payload).
__device__ __forceinline__ uint64_t record_bound(uint64_t k, const Header &h) {
  const uint64_t extra = (1u + h.offB > h.S * h.m) ? (1u + h.offB - h.S * h.m) : 0u;
  return (k + 7) / 8 + static_cast<uint64_t>(h.S) * k + extra * (k / h.m);
}

// Copy record bytes [src, src + n) into the warp's window so that the copy
// is 16-byte aligned on both sides: head and tail with plain loads, the
// middle with one TMA bulk copy.  Returns the shared address of byte 0.
__device__ __forceinline__ const uint8_t *stage_record(const uint8_t *src,
                                                       uint32_t n, uint8_t *win,
                                                       uint64_t *bar,
                                                       uint32_t &phase,
                                                       uint32_t lane, bool &ok) {
  const uint32_t mis = static_cast<uint32_t>(reinterpret_cast<uintptr_t>(src) & 15u);
  uint8_t *dst = win + mis;
  const uint32_t head = min(n, (16u - mis) & 15u);
  const uint32_t bulk = (n - head) & ~15u;
  if (bulk && lane == 0) {
    fence_proxy_async_smem();
    mbar_arrive_expect_tx(bar, bulk);
    bulk_g2s(dst + head, src + head, bulk, bar);
  }
  for (uint32_t i = lane; i < head; i += 32) dst[i] = src[i];
  for (uint32_t i = head + bulk + lane; i < n; i += 32) dst[i] = src[i];
  ok = true;
  if (bulk) {
    ok = mbar_wait_bounded(bar, phase);
    phase ^= 1u;
  }
  __syncwarp();
  return dst;
}

// 16 bytes of (a, b) starting at byte r (r uniform over the warp).
__device__ __forceinline__ uint4 bytes16(const uint4 &a, const uint4 &b, uint32_t r) {
  const uint32_t s = 8u * (r & 3u);
  uint32_t w0, w1, w2, w3, w4;
  switch (r >> 2) {
    case 0: w0 = a.x; w1 = a.y; w2 = a.z; w3 = a.w; w4 = b.x; break;
    case 1: w0 = a.y; w1 = a.z; w2 = a.w; w3 = b.x; w4 = b.y; break;
    case 2: w0 = a.z; w1 = a.w; w2 = b.x; w3 = b.y; w4 = b.z; break;
    default: w0 = a.w; w1 = b.x; w2 = b.y; w3 = b.z; w4 = b.w; break;
  }
  if (s == 0) return make_uint4(w0, w1, w2, w3);
  return make_uint4(__funnelshift_r(w0, w1, s), __funnelshift_r(w1, w2, s),
                    __funnelshift_r(w2, w3, s), __funnelshift_r(w3, w4, s));
}

// Warp copy of n bytes from shared src (any alignment, 16 bytes of slack
// readable past the end) to global dst, 16-byte stores where dst allows.
__device__ __forceinline__ void copy_s2g(uint8_t *dst, const uint8_t *src,
                                         uint32_t n, uint32_t lane) {
  const uint32_t head = min(
      n, (16u - static_cast<uint32_t>(reinterpret_cast<uintptr_t>(dst) & 15u)) & 15u);
  if (lane < head) dst[lane] = src[lane];
  const uint32_t body = (n - head) >> 4;
  const uint8_t *sb = src + head;
  const uint32_t r = static_cast<uint32_t>(reinterpret_cast<uintptr_t>(sb) & 15u);
  const uint4 *s16 = reinterpret_cast<const uint4 *>(sb - r);
  uint4 *d16 = reinterpret_cast<uint4 *>(dst + head);
  for (uint32_t j = lane; j < body; j += 32) d16[j] = bytes16(s16[j], s16[j + 1], r);
  const uint32_t done = head + 16u * body;
  for (uint32_t i = done + lane; i < n; i += 32) dst[i] = src[i];
}

__device__ __forceinline__ bool decode_chunk(const DecompressArgs &A,
                                             const Header &h, uint32_t c,
                                             uint64_t records_at,
                                             uint32_t *ring, uint32_t rmask,
                                             uint8_t *win, uint64_t *bar,
                                             uint32_t &phase, uint32_t lane) {
  const uint8_t *in = A.in;
  const uint8_t *table = in + kHeaderBytes;
  const uint8_t *index = table + 8ull * h.nc;
  const uint32_t j = c / kIndexStride;
  const uint64_t idxv = ld_le(index + 8ull * j, 8);
  const uint64_t part = record_bytes(table, j * kIndexStride, c, lane);
  bool bad = false;
  if (c == 0) bad = idxv != 0;
  if (c % kIndexStride == 0 && c > 0) {
    const uint64_t prev = ld_le(index + 8ull * (j - 1), 8);
    const uint64_t sb = record_bytes(table, c - kIndexStride, c, lane);
    bad = bad || prev + sb != idxv;
  }
  const uint32_t ntok = static_cast<uint32_t>(ld_le(table + 8ull * c, 4));
  const uint32_t pay = static_cast<uint32_t>(ld_le(table + 8ull * c + 4, 4));
  const uint64_t fb = (static_cast<uint64_t>(ntok) + 7) / 8;
  const uint64_t rec_at = records_at + idxv + part;
  const uint64_t chunk_at = static_cast<uint64_t>(c) * h.C;
  const uint32_t bytes_c = static_cast<uint32_t>((c + 1 < h.nc) ? h.C : h.n - chunk_at);
  const uint32_t k = bytes_c / h.S;
  const uint32_t tail = bytes_c - k * h.S;  // version 2, last chunk: bytes after the last symbol
  // version 2: a token count of 0 marks a stored chunk (its bytes as they are)
  const bool stored = h.version == 2 && ntok == 0;
  bad = bad || idxv > A.in_bytes || rec_at + fb + pay > A.in_bytes ||
        rec_at + fb + pay < rec_at || ntok > k || (ntok == 0 && !stored) ||
        (stored && pay != bytes_c) || (!stored && pay < tail) ||
        fb + pay > record_bound(k, h) + tail;
  if (bad) {
    if (lane == 0) atomicOr(A.err, kErrCorrupt);
    return true;
  }
  const uint8_t *flags = in + rec_at;  // read in place when there is no window
  if (win) {
    bool staged;
    flags = stage_record(in + rec_at, static_cast<uint32_t>(fb + pay), win, bar, phase,
                         lane, staged);
    if (!staged) {
      if (lane == 0) atomicOr(A.err, kErrTimeout);
      return false;
    }
  }
  const uint8_t *payload = flags + fb;
  uint8_t *dst = A.out + chunk_at;
  if (stored) {
    if (win) {
      copy_s2g(dst, payload, pay, lane);  // the window has slack past the record
    } else {
      for (uint32_t i = lane; i < pay; i += 32) dst[i] = payload[i];
    }
    return true;
  }
  const uint32_t S = h.S, offB = h.offB, tsz = 1 + h.offB;
  if (win) {
    // a chunk without pointers is its payload: copy it straight out
    uint32_t any = 0;
    for (uint32_t i = lane; i < fb; i += 32) any |= flags[i];
    if (!__any_sync(kFull, any != 0)) {
      if (ntok != k || pay != bytes_c) {
        if (lane == 0) atomicOr(A.err, kErrCorrupt);
        return true;
      }
      copy_s2g(dst, flags + fb, pay, lane);
      return true;
    }
  }
  const bool aligned = A.out_aligned != 0;
  const uint32_t lt = lanemask_lt(lane);

  uint32_t pos = 0;       // symbols produced
  uint64_t pay_used = 0;  // payload bytes consumed
  const uint32_t pay_tok = pay - tail;  // the tokens' payload; the tail follows it
  for (uint32_t tb = 0; tb < ntok; tb += 32) {
    const uint32_t t = tb + lane;
    const bool valid = t < ntok;
    const bool ism = valid && ((flags[t >> 3] >> (t & 7)) & 1u);
    const uint32_t mm = __ballot_sync(kFull, ism);
    const uint32_t vm = __ballot_sync(kFull, valid);
    const uint32_t nmb = __popc(mm & lt);
    const uint32_t nlb = __popc(vm & ~mm & lt);
    const uint64_t my_off = pay_used + S * nlb + tsz * nmb;
    const uint32_t my_sz = ism ? tsz : (valid ? S : 0u);
    bool tbad = valid && my_off + my_sz > pay_tok;
    uint32_t len = valid ? 1u : 0u, off = 0, val = 0;
    if (valid && !tbad) {
      if (ism) {
        len = payload[my_off];
        off = payload[my_off + 1];
        if (offB == 2) off |= static_cast<uint32_t>(payload[my_off + 2]) << 8;
        off += 1;
      } else {
        val = static_cast<uint32_t>(ld_le(payload + my_off, S));
      }
    }
    tbad = tbad || (ism && (len == 0 || off > h.W || (len > off && !h.overlap)));
    // inclusive scan of token lengths -> output start of each token
    uint32_t x = len;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(kFull, x, o);
      if (lane >= static_cast<uint32_t>(o)) x += y;
    }
    const uint32_t group_len = __shfl_sync(kFull, x, 31);
    const uint32_t start = pos + x - len;
    tbad = tbad || (ism && off > start);
    tbad = tbad || pos + group_len > k;
    if (__any_sync(kFull, tbad)) {
      if (lane == 0) atomicOr(A.err, kErrCorrupt);
      return true;
    }
    const uint32_t end = pos + group_len;
    if (mm == 0) {
      // all literals: lane i produces symbol pos + i
      if (valid) {
        ring[(pos + lane) & rmask] = val;
        store_symbol(dst + static_cast<uint64_t>(pos + lane) * S, val, S, aligned);
      }
    } else {
      const uint32_t start_key = valid ? start : kFull;
      for (uint32_t r0 = pos; r0 < end; r0 += 32) {
        const uint32_t jp = r0 + lane;
        const bool active = jp < end;
        // owning token: the last lane whose start is <= jp
        uint32_t lo = 0;
#pragma unroll
        for (uint32_t step = 16; step > 0; step >>= 1) {
          const uint32_t s = __shfl_sync(kFull, start_key, lo + step);
          if (s <= jp) lo += step;
        }
        const uint32_t o_ism = __shfl_sync(kFull, ism ? 1u : 0u, lo);
        const uint32_t o_off = __shfl_sync(kFull, off, lo);
        const uint32_t o_val = __shfl_sync(kFull, val, lo);
        uint32_t f = (active && o_ism) ? jp - o_off : jp;
        // resolve sources inside these 32 positions by pointer jumping
#pragma unroll
        for (int it = 0; it < 5; ++it) {
          const uint32_t src_lane = f >= r0 ? f - r0 : lane;
          const uint32_t g = __shfl_sync(kFull, f, src_lane);
          if (f >= r0) f = g;
        }
        const uint32_t v_here = __shfl_sync(kFull, o_val, f >= r0 ? f - r0 : lane);
        const uint32_t v = f >= r0 ? v_here : ring[f & rmask];
        __syncwarp();
        if (active) {
          ring[jp & rmask] = v;
          store_symbol(dst + static_cast<uint64_t>(jp) * S, v, S, aligned);
        }
        __syncwarp();
      }
    }
    __syncwarp();
    pos = end;
    pay_used += S * __popc(vm & ~mm) + tsz * __popc(mm);
  }
  if (pos != k || pay_used != pay_tok) {
    if (lane == 0) atomicOr(A.err, kErrCorrupt);
  } else if (lane < tail) {
    dst[static_cast<uint64_t>(k) * S + lane] = payload[pay_tok + lane];
  }
  return true;
}

}  // namespace

__global__ void __launch_bounds__(256) decompress_kernel(const DecompressArgs A) {
  extern __shared__ __align__(128) uint8_t smem[];
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t warp = threadIdx.x >> 5;
  const uint32_t wpb = blockDim.x >> 5;

  Header h;
  const bool ok = read_header(A.in, h);
  const bool leader = blockIdx.x == 0 && threadIdx.x == 0;
  if (!ok) {
    if (leader) atomicOr(A.err, kErrCorrupt);
    return;
  }
  if (h.n > A.out_cap) {
    if (leader) atomicOr(A.err, kErrSmall);
    return;
  }
  const uint64_t records_at = kHeaderBytes + 8ull * h.nc +
                              8ull * ((h.nc + kIndexStride - 1) / kIndexStride);
  if (records_at > A.in_bytes) {
    if (leader) atomicOr(A.err, kErrCorrupt);
    return;
  }
  if (leader) *A.out_bytes = h.n;
  // per-warp slice, decided from the header: mbarrier, a ring of >= W + 32
  // decoded symbols (offsets are at most W), and a window for one record
  uint32_t ring_n = 64;
  while (ring_n < h.W + 32) ring_n <<= 1;
  const uint32_t rmask = ring_n - 1;
  const uint64_t kfull = h.C / h.S;
  uint64_t need = 16 + 4ull * ring_n + ((record_bound(kfull, h) + 32 + 15) & ~15ull);
  // a record too large for one warp's window is read from global memory
  const bool windowed = need <= A.smem_bytes;
  if (!windowed) need = 16 + 4ull * ring_n;
  const uint64_t fit = A.smem_bytes / need;
  const uint32_t active = fit < wpb ? static_cast<uint32_t>(fit) : wpb;
  if (warp >= active) return;
  uint8_t *ws = smem + warp * need;
  uint64_t *bar = reinterpret_cast<uint64_t *>(ws);
  uint32_t *ring = reinterpret_cast<uint32_t *>(ws + 16);
  uint8_t *win = windowed ? ws + 16 + 4ull * ring_n : nullptr;
  if (lane == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
  }
  __syncwarp();
  uint32_t phase = 0;

  const uint32_t gw = blockIdx.x * active + warp;
  const uint32_t nwarps = gridDim.x * active;
  for (uint32_t c = gw; c < h.nc; c += nwarps)
    if (!decode_chunk(A, h, c, records_at, ring, rmask, win, bar, phase, lane)) break;
}

// Batched decompression: chunks of all streams in order, grid-stride; each
// warp finds its stream by a 32-way search over the streams' first chunks.
__global__ void __launch_bounds__(256) decompress_batch_kernel(const DecompressBatchArgs B) {
  extern __shared__ __align__(128) uint8_t smem[];
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t warp = threadIdx.x >> 5;
  const uint32_t wpb = blockDim.x >> 5;
  if (blockIdx.x == 0) {  // zero-byte streams: check the header, size 0
    for (uint32_t i = threadIdx.x; i < B.n_empty; i += blockDim.x) {
      Header h;
      if (!read_header(B.empties[i].in, h) || h.n != 0) atomicOr(B.err, kErrCorrupt);
      *B.empties[i].out_bytes = 0;
    }
  }
  const uint64_t need = 16 + 4ull * B.ring_n + B.win_bytes;
  const uint64_t fit = B.smem_bytes / need;
  const uint32_t active = fit < wpb ? static_cast<uint32_t>(fit) : wpb;
  if (warp >= active) return;
  uint8_t *ws = smem + warp * need;
  uint64_t *bar = reinterpret_cast<uint64_t *>(ws);
  uint32_t *ring = reinterpret_cast<uint32_t *>(ws + 16);
  uint8_t *win = ws + 16 + 4ull * B.ring_n;
  if (lane == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
  }
  __syncwarp();
  uint32_t phase = 0;
  const uint64_t stride = static_cast<uint64_t>(gridDim.x) * active;
  for (uint64_t g = static_cast<uint64_t>(blockIdx.x) * active + warp; g < B.total_chunks;
       g += stride) {
    uint32_t lo = 0, hi = B.n_items;
    while (hi - lo > 1) {
      const uint32_t step = (hi - lo + 31) / 32;
      const uint32_t idx = lo + lane * step;
      const bool le = idx < hi && B.item_base[idx] <= g;
      const uint32_t cnt = __popc(__ballot_sync(kFull, le));
      const uint32_t nlo = lo + (cnt - 1) * step;
      hi = min(hi, nlo + step);
      lo = nlo;
    }
    const DecItem it = B.items[lo];
    const uint32_t c = static_cast<uint32_t>(g - it.gbase);
    Header h{};
    const bool ok = it.in_bytes >= kHeaderBytes && read_header(it.in, h);
    const uint64_t records_at = kHeaderBytes + 8ull * h.nc +
                                8ull * ((h.nc + kIndexStride - 1) / kIndexStride);
    uint32_t ring_need = 64;
    while (ring_need < h.W + 32) ring_need <<= 1;
    // the header must still be the one the plan sized the slices for
    const bool fits = ok && h.nc == it.nc && ring_need <= B.ring_n &&
                      record_bound(h.C / h.S, h) + 32 <= B.win_bytes &&
                      records_at <= it.in_bytes && h.n <= it.out_cap;
    if (!fits) {
      if (lane == 0) atomicOr(B.err, h.n > it.out_cap && ok ? kErrSmall : kErrCorrupt);
      continue;
    }
    if (c == 0 && lane == 0) *it.out_bytes = h.n;
    DecompressArgs A{};
    A.in = it.in;
    A.in_bytes = it.in_bytes;
    A.out = it.out;
    A.out_cap = it.out_cap;
    A.out_bytes = it.out_bytes;
    A.err = B.err;
    A.out_aligned = static_cast<int>(it.out_aligned);
    if (!decode_chunk(A, h, c, records_at, ring, B.ring_n - 1, win, bar, phase, lane)) break;
  }
}

cudaError_t launch_decompress_batch(DecompressBatchArgs B, int block, cudaStream_t stream) {
  static std::mutex mu;
  static int per_sm = 0, sms = 0, cached_block = -1;
  static uint32_t cached_smem = 0;
  const size_t smem = B.smem_bytes;
  {
    std::lock_guard<std::mutex> lock(mu);
    if (cached_block != block || cached_smem != B.smem_bytes) {
      cudaError_t e = cudaFuncSetAttribute(decompress_batch_kernel,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           static_cast<int>(smem));
      if (e != cudaSuccess) return e;
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, decompress_batch_kernel,
                                                        block, smem);
      if (e != cudaSuccess) return e;
      int dev = 0;
      e = cudaGetDevice(&dev);
      if (e != cudaSuccess) return e;
      e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
      if (e != cudaSuccess) return e;
      cached_block = block;
      cached_smem = B.smem_bytes;
    }
  }
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  const uint64_t warps = block / 32;
  uint64_t want = (B.total_chunks + warps - 1) / warps;
  if (want == 0) want = 1;
  const uint64_t cap = static_cast<uint64_t>(per_sm) * sms;
  const unsigned grid = static_cast<unsigned>(want < cap ? want : cap);
  decompress_batch_kernel<<<grid, block, smem, stream>>>(B);
  return cudaGetLastError();
}

// Shared memory per block; each warp takes a slice sized from the header.
constexpr uint32_t kDecodeSmemPerBlock = 72 * 1024;

cudaError_t launch_decompress(DecompressArgs A, int block, cudaStream_t stream) {
  static std::mutex mu;
  static int per_sm = 0, sms = 0, cached_block = -1;
  A.smem_bytes = kDecodeSmemPerBlock;
  const size_t smem = kDecodeSmemPerBlock;
  {
    std::lock_guard<std::mutex> lock(mu);
    if (cached_block != block) {
      cudaError_t e = cudaFuncSetAttribute(
          decompress_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
          static_cast<int>(smem));
      if (e != cudaSuccess) return e;
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, decompress_kernel,
                                                        block, smem);
      if (e != cudaSuccess) return e;
      int dev = 0;
      e = cudaGetDevice(&dev);
      if (e != cudaSuccess) return e;
      e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
      if (e != cudaSuccess) return e;
      cached_block = block;
    }
  }
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  // enough blocks for the largest stream the input could hold, capped at the
  // resident limit (the grid cannot depend on the header: it is on the GPU)
  const uint64_t max_chunks = A.in_bytes / kTableEntry + 1;
  const uint64_t warps = block / 32;
  const uint64_t want = (max_chunks + warps - 1) / warps;
  const uint64_t cap = static_cast<uint64_t>(per_sm) * sms;
  const unsigned grid = static_cast<unsigned>(want < cap ? want : cap);
  decompress_kernel<<<grid, block, smem, stream>>>(A);
  return cudaGetLastError();
}

}  // namespace glz
