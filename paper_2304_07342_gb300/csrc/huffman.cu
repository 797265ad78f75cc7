// huffman.cu -- the Huffman stage that follows LZSS in the paper's use case
// (section 4.5: cuSZ Huffman-codes what gpuLZ produces).  Byte alphabet,
// an optimal prefix code limited to kHufMaxLen bits, canonical codes, and
// the "GHF1" stream described in include/lz.h.
//
//   huff_hist_kernel    256-bin histogram of the input
//   huff_book_kernel    one block: package-merge with every list built in
//                       parallel (each item finds its place in the merged
//                       list by a binary search in the other list), the
//                       selection walked level by level, canonical codes;
//                       writes the header and the code book
//   huff_sizes_kernel   one warp per 32 KiB block, one lane per 1 KiB
//                       sub-block: code bits per sub-block, their offsets
//   huff_scan_kernel    one block: block end offsets, stream size, capacity
//   huff_encode_kernel  one warp per block: each lane packs its sub-block's
//                       codes most significant bit first into 32-bit words
//                       (words shared with a neighbour lane by atomicOr)
//   huff_decode_kernel  one warp per block, one lane per sub-block: a
//                       4096-entry table in shared memory maps the next 12
//                       bits to (symbol, length)
#include <cuda_runtime.h>

#include <cstdint>

#include "glz_common.h"
#include "glz_device.cuh"

namespace glz {

namespace {

constexpr uint32_t kHufMaxLen = 12;
constexpr uint32_t kHufBlock = 32768;
constexpr uint32_t kHufSub = 1024;
constexpr uint32_t kHufSubs = kHufBlock / kHufSub;  // 32: one per lane
constexpr uint32_t kHufLengthsAt = 16;
constexpr uint32_t kHufTableAt = 272;
constexpr uint32_t kHufInvalid = 0xFFFFu;

__host__ __device__ __forceinline__ uint64_t huf_subs_at(uint64_t nb) {
  return kHufTableAt + 8ull * nb;
}
__host__ __device__ __forceinline__ uint64_t huf_bits_at(uint64_t nb) {
  return kHufTableAt + 8ull * nb + 4ull * kHufSubs * nb;
}

__device__ __forceinline__ uint64_t ld_u64_le(const uint8_t *p) {
  uint64_t v = 0;
  for (int i = 0; i < 8; ++i) v |= static_cast<uint64_t>(p[i]) << (8 * i);
  return v;
}

// ---- histogram -----------------------------------------------------------------

__global__ void __launch_bounds__(256) huff_hist_kernel(const uint8_t *in, uint64_t n,
                                                       unsigned long long *hist) {
  __shared__ uint32_t h[8][256];  // one copy per warp: fewer same-address collisions
  for (uint32_t i = threadIdx.x; i < 8 * 256; i += blockDim.x) (&h[0][0])[i] = 0;
  __syncthreads();
  uint32_t *mine = h[threadIdx.x >> 5];
  const uint64_t mis = (4u - (reinterpret_cast<uintptr_t>(in) & 3u)) & 3u;
  const uint64_t head = n < mis ? n : mis;
  const uint64_t words = (n - head) / 4;
  const uint32_t *w32 = reinterpret_cast<const uint32_t *>(in + head);
  const uint64_t tid = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  const uint64_t stride = static_cast<uint64_t>(gridDim.x) * blockDim.x;
  for (uint64_t i = tid; i < words; i += stride) {
    const uint32_t v = w32[i];
    atomicAdd(&mine[v & 0xFF], 1u);
    atomicAdd(&mine[(v >> 8) & 0xFF], 1u);
    atomicAdd(&mine[(v >> 16) & 0xFF], 1u);
    atomicAdd(&mine[v >> 24], 1u);
  }
  if (tid < head) atomicAdd(&mine[in[tid]], 1u);
  const uint64_t done = head + 4 * words;
  if (tid < n - done) atomicAdd(&mine[in[done + tid]], 1u);
  __syncthreads();
  for (uint32_t s = threadIdx.x; s < 256; s += blockDim.x) {
    uint32_t t = 0;
    for (int w = 0; w < 8; ++w) t += h[w][s];
    if (t) atomicAdd(&hist[s], static_cast<unsigned long long>(t));
  }
}

// ---- code book -------------------------------------------------------------------

// Canonical codes of lengths len[256] (one thread per symbol, blockDim >= 256):
// symbols in order of (length, value) take consecutive values, shifted left
// when the length grows.  first[] and cnt[] are shared scratch.
__device__ void canonical_codes(const uint32_t *len, uint32_t *first, uint32_t *cnt,
                                uint32_t *code_out) {
  const uint32_t t = threadIdx.x;
  if (t <= kHufMaxLen) cnt[t] = 0;
  __syncthreads();
  if (t < 256 && len[t]) atomicAdd(&cnt[len[t]], 1u);
  __syncthreads();
  if (t == 0) {
    uint32_t next = 0;
    for (uint32_t l = 1; l <= kHufMaxLen; ++l) {
      first[l] = next;
      next = (next + cnt[l]) << 1;
    }
  }
  __syncthreads();
  if (t < 256) {
    const uint32_t l = len[t];
    uint32_t rank = 0;
    if (l)
      for (uint32_t s = 0; s < t; ++s) rank += len[s] == l;
    code_out[t] = l ? first[l] + rank : 0;
  }
  __syncthreads();
}

// Package-merge over the present symbols (at most 256, so every list has at
// most 511 items): leaves sorted by (count, value); list d (d = 0 the
// shallowest) merges the leaves with the packages of consecutive pairs of
// list d + 1, by weight, a leaf before a package of equal weight; the first
// 2n - 2 items of list 0 are selected and a selected package selects its two
// children.  A symbol's length is the number of lists where it is selected.
__global__ void __launch_bounds__(512) huff_book_kernel(const unsigned long long *hist,
                                                       uint64_t n_bytes, uint8_t *out,
                                                       uint32_t *book) {
  __shared__ unsigned long long hw[256], leafw[256];
  __shared__ unsigned long long w[2][512];
  __shared__ uint16_t ref[kHufMaxLen][512];  // 0x8000 | symbol, or package index
  __shared__ uint8_t sel[kHufMaxLen][512];
  __shared__ uint32_t leafsym[256], len[256], code[256], first[kHufMaxLen + 1],
      cnt[kHufMaxLen + 1], count[kHufMaxLen];
  const uint32_t t = threadIdx.x;
  if (t < 256) {
    hw[t] = hist[t];
    len[t] = 0;
  }
  for (uint32_t i = t; i < kHufMaxLen * 512; i += blockDim.x) (&sel[0][0])[i] = 0;
  __syncthreads();
  const uint32_t n = __syncthreads_count(t < 256 && hw[t] > 0);
  if (n == 1) {
    if (t < 256 && hw[t]) len[t] = 1;
  } else if (n > 1) {
    if (t < 256 && hw[t]) {
      uint32_t r = 0;
      for (uint32_t s = 0; s < 256; ++s)
        r += hw[s] && (hw[s] < hw[t] || (hw[s] == hw[t] && s < t));
      leafsym[r] = t;
      leafw[r] = hw[t];
    }
    __syncthreads();
    const uint32_t deep = kHufMaxLen - 1;
    if (t < n) {
      w[deep & 1][t] = leafw[t];
      ref[deep][t] = static_cast<uint16_t>(0x8000u | leafsym[t]);
    }
    if (t == 0) count[deep] = n;
    __syncthreads();
    for (int d = static_cast<int>(deep) - 1; d >= 0; --d) {
      const unsigned long long *below = w[(d + 1) & 1];
      unsigned long long *cur = w[d & 1];
      const uint32_t np = count[d + 1] / 2;
      if (t < n) {
        // leaf t: after every package strictly lighter
        const unsigned long long x = leafw[t];
        uint32_t lo = 0, hi = np;
        while (lo < hi) {
          const uint32_t mid = (lo + hi) / 2;
          if (below[2 * mid] + below[2 * mid + 1] < x) lo = mid + 1;
          else hi = mid;
        }
        cur[t + lo] = x;
        ref[d][t + lo] = static_cast<uint16_t>(0x8000u | leafsym[t]);
      } else if (t < n + np) {
        // package j: after every leaf of equal or smaller weight
        const uint32_t j = t - n;
        const unsigned long long x = below[2 * j] + below[2 * j + 1];
        uint32_t lo = 0, hi = n;
        while (lo < hi) {
          const uint32_t mid = (lo + hi) / 2;
          if (leafw[mid] <= x) lo = mid + 1;
          else hi = mid;
        }
        cur[j + lo] = x;
        ref[d][j + lo] = static_cast<uint16_t>(j);
      }
      if (t == 0) count[d] = n + np;
      __syncthreads();
    }
    for (uint32_t i = t; i < count[0] && i < 2 * n - 2; i += blockDim.x) sel[0][i] = 1;
    for (uint32_t d = 0; d < kHufMaxLen; ++d) {
      __syncthreads();
      for (uint32_t i = t; i < count[d]; i += blockDim.x) {
        if (!sel[d][i]) continue;
        const uint32_t r = ref[d][i];
        if (r & 0x8000u) {
          atomicAdd(&len[r & 0xFFu], 1u);
        } else if (d + 1 < kHufMaxLen) {
          sel[d + 1][2 * r] = 1;
          sel[d + 1][2 * r + 1] = 1;
        }
      }
    }
  }
  __syncthreads();
  canonical_codes(len, first, cnt, code);
  if (t < 256) {
    book[t] = code[t] | (len[t] << 24);
    out[kHufLengthsAt + t] = static_cast<uint8_t>(len[t]);
  }
  if (t < 16) {
    uint32_t b = 0;
    if (t < 4) b = "GHF1"[t];
    else if (t < 8) b = (kHufBlock >> (8 * (t - 4))) & 0xFF;
    else b = static_cast<uint32_t>(n_bytes >> (8 * (t - 8))) & 0xFF;
    out[t] = static_cast<uint8_t>(b);
  }
}

// ---- encode ------------------------------------------------------------------------

// This lane's sub-block of block b: [lo, hi) of the input (empty past n).
__device__ __forceinline__ void sub_range(uint64_t b, uint32_t lane, uint64_t n, uint64_t &lo,
                                          uint64_t &hi) {
  lo = b * kHufBlock + static_cast<uint64_t>(lane) * kHufSub;
  hi = lo + kHufSub < n ? lo + kHufSub : n;
  if (lo > n) lo = n;
}

// The 32 bytes of sub-block s of block b that lane `lane` handles, as eight
// little-endian words (zero past hi); 16-byte loads when `in` is aligned.
__device__ __forceinline__ void lane_bytes(const uint8_t *in, uint64_t at, uint64_t hi,
                                           bool in16, uint32_t (&w)[8]) {
  if (in16 && at + 32 <= hi) {
    const uint4 a = *reinterpret_cast<const uint4 *>(in + at);
    const uint4 c = *reinterpret_cast<const uint4 *>(in + at + 16);
    w[0] = a.x; w[1] = a.y; w[2] = a.z; w[3] = a.w;
    w[4] = c.x; w[5] = c.y; w[6] = c.z; w[7] = c.w;
  } else {
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      uint32_t v = 0;
      for (int k = 0; k < 4; ++k) {
        const uint64_t idx = at + 4 * q + k;
        if (idx < hi) v |= static_cast<uint32_t>(in[idx]) << (8 * k);
      }
      w[q] = v;
    }
  }
}

// Code bits of each sub-block and their offsets inside the block.  One
// warp per block; for each sub-block the lanes read 32 consecutive bytes
// each (coalesced) and the warp sums their code lengths.
__global__ void __launch_bounds__(256) huff_sizes_kernel(const uint8_t *in, uint64_t n,
                                                        uint8_t *out, const uint32_t *book) {
  __shared__ uint8_t len[256];
  for (uint32_t s = threadIdx.x; s < 256; s += blockDim.x) len[s] = book[s] >> 24;
  __syncthreads();
  const uint32_t lane = threadIdx.x & 31;
  const uint64_t nb = (n + kHufBlock - 1) / kHufBlock;
  const uint64_t gw = (static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const uint64_t nw = (static_cast<uint64_t>(gridDim.x) * blockDim.x) >> 5;
  uint32_t *subs = reinterpret_cast<uint32_t *>(out + huf_subs_at(nb));
  unsigned long long *table = reinterpret_cast<unsigned long long *>(out + kHufTableAt);
  const bool in16 = (reinterpret_cast<uintptr_t>(in) & 15u) == 0;
  for (uint64_t b = gw; b < nb; b += nw) {
    uint32_t mine = 0;  // bits of sub-block `lane`
    for (uint32_t sb = 0; sb < kHufSubs; ++sb) {
      uint64_t lo, hi;
      sub_range(b, sb, n, lo, hi);
      if (lo >= hi) break;  // every later sub-block is empty too
      uint32_t w[8];
      lane_bytes(in, lo + 32ull * lane, hi, in16, w);
      const uint32_t valid = lo + 32ull * lane >= hi ? 0u
                             : static_cast<uint32_t>(min(hi - lo - 32ull * lane, 32ull));
      uint32_t bits = 0;
#pragma unroll
      for (int q = 0; q < 8; ++q)
#pragma unroll
        for (int k = 0; k < 4; ++k)
          bits += (4u * q + k < valid) ? len[(w[q] >> (8 * k)) & 0xFF] : 0u;
      const uint32_t total = __reduce_add_sync(kFull, bits);
      if (lane == sb) mine = total;
    }
    uint32_t incl = mine;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(kFull, incl, o);
      if (lane >= static_cast<uint32_t>(o)) incl += y;
    }
    subs[b * kHufSubs + lane] = incl - mine;
    const uint32_t total = __shfl_sync(kFull, incl, 31);
    if (lane == 0) table[b] = static_cast<unsigned long long>((total + 31) / 32) * 4;  // size
  }
}

// Block sizes -> block end offsets (inclusive prefix sums), the stream size
// and the capacity check.  One block of 1024 threads; thread t scans a run
// of consecutive entries.
__global__ void __launch_bounds__(1024) huff_scan_kernel(uint8_t *out, uint64_t n,
                                                        uint64_t out_cap,
                                                        unsigned long long *out_bytes,
                                                        uint32_t *err) {
  __shared__ unsigned long long part[1024];
  const uint64_t nb = (n + kHufBlock - 1) / kHufBlock;
  unsigned long long *table = reinterpret_cast<unsigned long long *>(out + kHufTableAt);
  const uint32_t t = threadIdx.x;
  const uint64_t per = (nb + blockDim.x - 1) / blockDim.x;
  const uint64_t lo = t * per < nb ? t * per : nb;
  const uint64_t hi = lo + per < nb ? lo + per : nb;
  unsigned long long s = 0;
  for (uint64_t b = lo; b < hi; ++b) s += table[b];
  part[t] = s;
  __syncthreads();
  for (uint32_t o = 1; o < blockDim.x; o <<= 1) {  // inclusive scan of the runs
    const unsigned long long y = t >= o ? part[t - o] : 0ull;
    __syncthreads();
    part[t] += y;
    __syncthreads();
  }
  unsigned long long run = part[t] - s;
  for (uint64_t b = lo; b < hi; ++b) {
    run += table[b];
    table[b] = run;
  }
  if (t == blockDim.x - 1) {
    const unsigned long long total = huf_bits_at(nb) + part[t];
    *out_bytes = total;
    if (total > out_cap) atomicOr(err, kErrSmall);
  }
}

// Encoding, one warp per block.  Sub-block by sub-block, each lane codes
// 32 consecutive bytes; a warp scan of the lanes' bit counts places each
// lane's codes, which are ORed into a per-warp shared-memory copy of the
// sub-block's words.  The complete words go out with coalesced stores; a
// last, partial word carries over to the next sub-block (or is written at
// the end of the block), so every word of the bit string is written once.
constexpr uint32_t kEncWords = (kHufSub * kHufMaxLen) / 32 + 2;  // words of one sub-block

__global__ void __launch_bounds__(256) huff_encode_kernel(const uint8_t *in, uint64_t n,
                                                         uint8_t *out, uint64_t out_cap,
                                                         const uint32_t *book) {
  __shared__ uint32_t cl[256];  // code | length << 24
  __shared__ uint32_t sbuf[8][kEncWords];
  for (uint32_t s = threadIdx.x; s < 256; s += blockDim.x) cl[s] = book[s];
  __syncthreads();
  const uint32_t lane = threadIdx.x & 31;
  uint32_t *wb = sbuf[threadIdx.x >> 5];
  const uint64_t nb = (n + kHufBlock - 1) / kHufBlock;
  const uint64_t gw = (static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const uint64_t nw = (static_cast<uint64_t>(gridDim.x) * blockDim.x) >> 5;
  const uint64_t bits_at = huf_bits_at(nb);
  const uint32_t *subs = reinterpret_cast<const uint32_t *>(out + huf_subs_at(nb));
  const unsigned long long *table =
      reinterpret_cast<const unsigned long long *>(out + kHufTableAt);
  const bool in16 = (reinterpret_cast<uintptr_t>(in) & 15u) == 0;
  for (uint64_t b = gw; b < nb; b += nw) {
    const uint64_t start = b ? table[b - 1] : 0ull, end = table[b];
    if (bits_at + end > out_cap) continue;  // reported by the scan kernel
    uint32_t *w32 = reinterpret_cast<uint32_t *>(out + bits_at + start);
    uint32_t carry = 0;     // bits already placed in word `at / 32` (the partial word)
    uint32_t at = 0;        // bit position in the block after the last sub-block
    for (uint32_t sb = 0; sb < kHufSubs; ++sb) {
      uint64_t lo, hi;
      sub_range(b, sb, n, lo, hi);
      if (lo >= hi) break;
      const uint32_t a = subs[b * kHufSubs + sb];  // == at
      uint32_t w[8];
      lane_bytes(in, lo + 32ull * lane, hi, in16, w);
      const uint32_t valid = lo + 32ull * lane >= hi ? 0u
                             : static_cast<uint32_t>(min(hi - lo - 32ull * lane, 32ull));
      uint32_t bits = 0;
#pragma unroll
      for (int q = 0; q < 8; ++q)
#pragma unroll
        for (int k = 0; k < 4; ++k)
          bits += (4u * q + k < valid) ? (cl[(w[q] >> (8 * k)) & 0xFF] >> 24) : 0u;
      uint32_t incl = bits;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(kFull, incl, o);
        if (lane >= static_cast<uint32_t>(o)) incl += y;
      }
      const uint32_t sub_bits = __shfl_sync(kFull, incl, 31);
      const uint32_t r0 = a % 32;                      // bits of the carried word
      const uint32_t nwords = (r0 + sub_bits + 31) / 32;
      for (uint32_t k = lane; k < nwords; k += 32) wb[k] = 0;
      __syncwarp();
      if (lane == 0 && r0) wb[0] = carry;
      __syncwarp();
      // this lane's codes, most significant bit first, from bit r0 + excl
      uint32_t p = r0 + incl - bits;
      uint64_t acc = 0;
      uint32_t nacc = p % 32, wi = p / 32;
      bool first = true;
#pragma unroll
      for (int q = 0; q < 8; ++q)
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          if (4u * q + k < valid) {
            const uint32_t c = cl[(w[q] >> (8 * k)) & 0xFF];
            const uint32_t l = c >> 24;
            acc = (acc << l) | (c & 0xFFFFFFu);
            nacc += l;
            if (nacc >= 32) {
              nacc -= 32;
              const uint32_t word = static_cast<uint32_t>(acc >> nacc);
              if (first) atomicOr(&wb[wi], word);  // shared with the lane before
              else wb[wi] = word;
              first = false;
              ++wi;
              acc &= (1ull << nacc) - 1ull;
            }
          }
        }
      if (nacc > 0 && bits > 0) atomicOr(&wb[wi], static_cast<uint32_t>(acc << (32 - nacc)));
      __syncwarp();
      // complete words out; a partial last word stays for the next sub-block
      const uint32_t full = (r0 + sub_bits) / 32;
      for (uint32_t k = lane; k < full; k += 32) w32[a / 32 + k] = wb[k];
      carry = (r0 + sub_bits) % 32 ? wb[full] : 0u;
      __syncwarp();
      at = a + sub_bits;
    }
    if (at % 32 && lane == 0) w32[at / 32] = carry;  // the block's last, padded word
  }
}

// ---- decode ------------------------------------------------------------------------

struct HufHeader {
  uint64_t n, nb, bits_at;
  bool ok;
};

__device__ __forceinline__ HufHeader huf_header(const uint8_t *in, uint64_t in_bytes) {
  HufHeader h{};
  h.ok = in_bytes >= kHufTableAt && in[0] == 'G' && in[1] == 'H' && in[2] == 'F' &&
         in[3] == '1' && in[4] == (kHufBlock & 0xFF) && in[5] == ((kHufBlock >> 8) & 0xFF) &&
         in[6] == 0 && in[7] == 0;
  if (!h.ok) return h;
  h.n = ld_u64_le(in + 8);
  h.nb = (h.n + kHufBlock - 1) / kHufBlock;
  h.bits_at = huf_bits_at(h.nb);
  h.ok = h.nb < (1ull << 40) && h.bits_at <= in_bytes;
  return h;
}

__global__ void __launch_bounds__(256) huff_decode_kernel(const uint8_t *in, uint64_t in_bytes,
                                                         uint8_t *out, uint64_t out_cap,
                                                         unsigned long long *out_bytes,
                                                         uint32_t *err) {
  __shared__ uint16_t dec[1u << kHufMaxLen];  // symbol | length << 8
  __shared__ uint32_t len[256], code[256], first[kHufMaxLen + 1], cnt[kHufMaxLen + 1];
  __shared__ uint32_t bad_code;
  const uint32_t t = threadIdx.x;
  const HufHeader h = huf_header(in, in_bytes);
  if (!h.ok) {
    if (blockIdx.x == 0 && t == 0) atomicOr(err, kErrCorrupt);
    return;
  }
  if (h.n > out_cap) {
    if (blockIdx.x == 0 && t == 0) atomicOr(err, kErrSmall);
    return;
  }
  if (blockIdx.x == 0 && t == 0) *out_bytes = h.n;
  if (t == 0) bad_code = 0;
  for (uint32_t i = t; i < (1u << kHufMaxLen); i += blockDim.x) dec[i] = kHufInvalid;
  if (t < 256) len[t] = in[kHufLengthsAt + t];
  __syncthreads();
  // the lengths must form a complete code (or one symbol of length 1)
  uint32_t present = 0, kraft = 0;
  if (t < 256 && len[t]) {
    if (len[t] > kHufMaxLen) atomicOr(&bad_code, 1u);
    else kraft = 1u << (kHufMaxLen - len[t]);
    present = 1;
  }
  const uint32_t n_present = __syncthreads_count(present);
  __shared__ uint32_t kraft_sum;
  if (t == 0) kraft_sum = 0;
  __syncthreads();
  if (kraft) atomicAdd(&kraft_sum, kraft);
  __syncthreads();
  const bool complete = n_present == 1 ? kraft_sum == (1u << (kHufMaxLen - 1))
                                       : kraft_sum == (1u << kHufMaxLen);
  if (bad_code || (h.n > 0 && !complete)) {
    if (blockIdx.x == 0 && t == 0) atomicOr(err, kErrCorrupt);
    return;
  }
  canonical_codes(len, first, cnt, code);
  // symbols in canonical order: those of length l hold places off[l] ..
  // off[l] + cnt[l] - 1, by value
  __shared__ uint32_t off[kHufMaxLen + 2];
  __shared__ uint8_t order[256];
  if (t == 0) {
    off[1] = 0;
    for (uint32_t l = 1; l <= kHufMaxLen; ++l) off[l + 1] = off[l] + cnt[l];
  }
  __syncthreads();
  if (t < 256 && len[t]) order[off[len[t]] + code[t] - first[len[t]]] = static_cast<uint8_t>(t);
  __syncthreads();
  // entry e (the next 12 bits) belongs to the length l whose codes cover
  // e >> (12 - l); each thread fills 16 entries
  for (uint32_t e = t; e < (1u << kHufMaxLen); e += blockDim.x) {
    uint16_t v = kHufInvalid;
    for (uint32_t l = 1; l <= kHufMaxLen; ++l) {
      const uint32_t c = e >> (kHufMaxLen - l);
      if (cnt[l] && c >= first[l] && c - first[l] < cnt[l]) {
        v = static_cast<uint16_t>(order[off[l] + c - first[l]] | (l << 8));
        break;
      }
    }
    dec[e] = v;
  }
  __syncthreads();

  const uint32_t lane = t & 31;
  const uint64_t gw = (static_cast<uint64_t>(blockIdx.x) * blockDim.x + t) >> 5;
  const uint64_t nw = (static_cast<uint64_t>(gridDim.x) * blockDim.x) >> 5;
  const uint32_t *subs = reinterpret_cast<const uint32_t *>(in + huf_subs_at(h.nb));
  const uint8_t *table = in + kHufTableAt;
  const bool out16 = (reinterpret_cast<uintptr_t>(out) & 15u) == 0;
  for (uint64_t b = gw; b < h.nb; b += nw) {
    const uint64_t start = b ? ld_u64_le(table + 8 * (b - 1)) : 0ull;
    const uint64_t end = ld_u64_le(table + 8 * b);
    const uint64_t bytes = end - start;
    bool bad = end < start || bytes % 4 || h.bits_at + end > in_bytes || bytes > (1ull << 20);
    const uint32_t nbits = static_cast<uint32_t>(bytes * 8);
    uint64_t lo, hi;
    sub_range(b, lane, h.n, lo, hi);
    const uint32_t o = bad ? 0 : subs[b * kHufSubs + lane];
    const uint32_t o_down = __shfl_down_sync(kFull, o, 1);  // every lane takes part
    const uint32_t o_next = lane < 31 ? o_down : 0u;
    bad = bad || o > nbits || (lane == 0 && o != 0);
    if (__any_sync(kFull, bad)) {
      if (lane == 0) atomicOr(err, kErrCorrupt);
      continue;
    }
    const uint32_t *w32 = reinterpret_cast<const uint32_t *>(in + h.bits_at + start);
    const uint32_t nwords = static_cast<uint32_t>(bytes / 4);
    // bit buffer: the next `avail` (>= 32 after a refill) bits, left-aligned;
    // `nextw` is the word after them, loaded one refill ahead
    uint32_t wi = o / 32;
    uint64_t buf = (static_cast<uint64_t>(wi < nwords ? w32[wi] : 0u) << 32) |
                   (wi + 1 < nwords ? w32[wi + 1] : 0u);
    buf <<= o % 32;
    uint32_t avail = 64 - o % 32;
    wi += 2;
    uint32_t nextw = wi < nwords ? w32[wi] : 0u;
    uint32_t pos = o;
    bool invalid = false;
    auto next_symbol = [&]() -> uint32_t {
      const uint32_t e = dec[static_cast<uint32_t>(buf >> (64 - kHufMaxLen))];
      const uint32_t l = (e >> 8) & 15u;  // an invalid entry reads as length 15
      invalid |= e == kHufInvalid;
      buf <<= l;
      avail -= l;
      pos += l;
      if (avail < 32) {
        buf |= static_cast<uint64_t>(nextw) << (32 - avail);
        avail += 32;
        ++wi;
        nextw = wi < nwords ? w32[wi] : 0u;
      }
      return e & 0xFFu;
    };
    uint64_t i = lo;
    if (out16) {
      for (; i + 16 <= hi; i += 16) {
        uint32_t w[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          uint32_t v = next_symbol();
          v |= next_symbol() << 8;
          v |= next_symbol() << 16;
          v |= next_symbol() << 24;
          w[q] = v;
        }
        // streaming store: the output should not push the stream's lines,
        // which the other lanes of the warp still read, out of L2
        __stcs(reinterpret_cast<uint4 *>(out + i), make_uint4(w[0], w[1], w[2], w[3]));
      }
    }
    for (; i < hi; ++i) out[i] = static_cast<uint8_t>(next_symbol());
    // each sub-block ends where the next begins; the block's words hold
    // exactly the bits used, rounded up to a word
    bool lane_bad = invalid || pos > nbits;
    if (lane < 31) lane_bad = lane_bad || pos != o_next;
    else lane_bad = lane_bad || (pos + 31) / 32 != nwords;
    if (__any_sync(kFull, lane_bad) && lane == 0) atomicOr(err, kErrCorrupt);
  }
}

}  // namespace

cudaError_t launch_huff_compress(const uint8_t *in, uint64_t n, uint8_t *out, uint64_t out_cap,
                                 unsigned long long *out_bytes, unsigned long long *hist,
                                 uint32_t *book, uint32_t *err, int sms, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(hist, 0, 256 * sizeof(unsigned long long), st);
  if (e != cudaSuccess) return e;
  const uint64_t nb = (n + kHufBlock - 1) / kHufBlock;
  if (n) {
    huff_hist_kernel<<<sms * 4, 256, 0, st>>>(in, n, hist);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  huff_book_kernel<<<1, 512, 0, st>>>(hist, n, out, book);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (nb == 0) {
    huff_scan_kernel<<<1, 1024, 0, st>>>(out, n, out_cap, out_bytes, err);
    return cudaGetLastError();
  }
  const uint64_t warps = nb < static_cast<uint64_t>(sms) * 64 ? nb : static_cast<uint64_t>(sms) * 64;
  const unsigned grid = static_cast<unsigned>((warps + 7) / 8);
  huff_sizes_kernel<<<grid, 256, 0, st>>>(in, n, out, book);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  huff_scan_kernel<<<1, 1024, 0, st>>>(out, n, out_cap, out_bytes, err);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  huff_encode_kernel<<<grid, 256, 0, st>>>(in, n, out, out_cap, book);
  return cudaGetLastError();
}

cudaError_t launch_huff_decompress(const uint8_t *in, uint64_t in_bytes, uint8_t *out,
                                   uint64_t out_cap, unsigned long long *out_bytes,
                                   uint32_t *err, int sms, cudaStream_t st) {
  huff_decode_kernel<<<sms * 8, 256, 0, st>>>(in, in_bytes, out, out_cap, out_bytes, err);
  return cudaGetLastError();
}

uint64_t huff_layout_bits_at(uint64_t n) {
  return huf_bits_at((n + kHufBlock - 1) / kHufBlock);
}

}  // namespace glz
