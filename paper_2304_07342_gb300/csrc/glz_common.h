// glz_common.h -- launch-parameter structs shared by the host side of the
// C ABI and the kernels (product code only).
#pragma once

#include <cstdint>

namespace glz {

constexpr uint32_t kHeaderBytes = 32;   // GLZ1 header
constexpr uint32_t kTableEntry = 8;     // {u32 n_tokens, u32 payload_bytes}
constexpr uint32_t kIndexStride = 64;   // one u64 index entry per 64 chunks
constexpr uint32_t kMaxChunk = 32768;   // bytes
constexpr uint32_t kMaxWindow = 1024;   // symbols

// Matchers of the greedy parse (lz_match in lz.h).
constexpr uint32_t kMatchExact = 0;  // longest match, nearest offset on ties
constexpr uint32_t kMatchPaper = 1;  // the paper's forward scan (section 3.3.2)
constexpr uint32_t kMatchOverlap = 2;  // exact, a match may overlap its output

// Sticky device error bits (lz_sync maps them back to lz_status).
constexpr uint32_t kErrSmall = 1u << 0;
constexpr uint32_t kErrCorrupt = 1u << 1;
constexpr uint32_t kErrTimeout = 1u << 2;
constexpr uint32_t kErrInternal = 1u << 3;  // a device consistency check failed

// Bounded spins: a device wait that exceeds this many polls gives up and
// raises kErrTimeout instead of hanging the GPU.
constexpr uint32_t kSpinLimit = 1u << 22;

// Per-warp shared-memory layout of the compressor (byte offsets from the
// warp's slice; every region 16-byte aligned).
struct CompressSmem {
  uint32_t in_off;     // staged chunk, C bytes
  uint32_t prev_off;   // u16 per position: previous position, same key hash
  uint32_t flags_off;  // flag bits of up to k tokens
  uint32_t pay_off;    // payload staging (worst case); also the hash table
  uint32_t pay_bytes;  // size of the payload staging region
  uint32_t maybe_off;  // one bit per position: a match of >= m may exist
  uint32_t mbar_off;   // mbarrier for the TMA bulk copy
  uint32_t per_warp;   // total bytes per warp
  uint32_t hash_log2;  // hash table entries = 1 << hash_log2 (u16 each)
};

// One buffer to compress (one stream): per-buffer parameters and places.
struct BufDesc {
  const uint8_t *in;
  uint64_t n;
  uint8_t *out;
  uint64_t cap;
  unsigned long long *out_bytes;
  uint32_t S, C, W, m, M, offB;
  uint32_t nc;          // chunks
  uint32_t in_aligned;  // in is 16-byte aligned: TMA bulk staging
  uint32_t match;       // kMatchExact, kMatchPaper or kMatchOverlap
  uint32_t version;     // stream version written: 1, or 2 (stored chunks); 0 reads as 1
  uint64_t records_at;  // byte offset of the records region
  uint64_t gbase;       // index of this buffer's chunk 0 among all chunks
};

struct CompressArgs {
  BufDesc buf;                 // single-buffer launch
  const BufDesc *items;        // batched launch (nullptr for a single buffer)
  const uint64_t *item_base;   // items[i].gbase, ascending (batched launch)
  uint32_t n_items;            // non-empty items
  uint64_t total_chunks;       // chunks over all items
  CompressSmem sm;             // per-warp layout (covers every item)
  unsigned long long *status;  // one look-back word per chunk (cleared per call)
  uint32_t *ticket;            // work counter (cleared per call)
  uint32_t *err;               // sticky error bits
  uint8_t *park;               // parking slots: grid warps x park_slots
  uint32_t park_slots;         // slots per warp (<= 32)
  uint32_t park_slot_bytes;    // one worst-case record, 16-byte multiple
  uint32_t spin_limit;         // polls before a device wait gives up (kSpinLimit normally)
  uint32_t first_ticket;       // first chunk handed out (0 normally)
  uint32_t end_chunk;          // single buffer: chunks [first_ticket, end_chunk) are taken
};

// Placement of one shard stream inside a whole-input stream (lz_stitch).
struct StitchArgs {
  const uint8_t *shard;   // 8-byte aligned
  uint64_t shard_chunks;  // chunks in the shard
  uint64_t chunk_base;    // chunks before it (multiple of kIndexStride)
  uint64_t total_chunks;
  uint64_t total_bytes;
  uint64_t record_base;   // record bytes of the shards before it
  uint64_t src_records;   // byte offset of the shard's records
  uint64_t record_bytes;  // the shard's record bytes
  uint64_t dst_records;   // byte offset of this shard's records in out
  uint8_t *out;           // 8-byte aligned
  uint32_t *err;
};

struct DecompressArgs {
  const uint8_t *in;
  uint64_t in_bytes;
  uint8_t *out;
  uint64_t out_cap;
  unsigned long long *out_bytes;
  uint32_t *err;
  uint32_t smem_bytes;  // dynamic shared memory per block
  int out_aligned;      // out is 16-byte aligned
};

// One stream of a batched decompression.
struct DecItem {
  const uint8_t *in;
  uint64_t in_bytes;
  uint8_t *out;
  uint64_t out_cap;
  unsigned long long *out_bytes;
  uint64_t gbase;  // index of this stream's chunk 0 among all chunks
  uint32_t nc;
  uint32_t out_aligned;
};

// Per-warp shared-memory slice of the decoder (byte offsets, 16-byte
// aligned): an mbarrier, one mark byte per position of the chunk (0 inside
// a token, 1 where a literal starts, 2 where a pointer starts), a copy of
// the record's flag bytes, the high bytes of (offset - 1) when one-byte
// symbols carry two-byte offsets, then -- when they fit -- the io area:
// the chunk's output image from its start, with the record staged at its
// end.  When no pointer takes more payload bytes than the symbols it
// covers (S * m >= 1 + offB for every stream; `shared`), the output
// written so far never reaches a payload byte not yet read, so the area
// only needs room for the larger of the two; otherwise it holds both side
// by side.  Without the io area (`staged` false) a warp decodes straight
// into the output buffer and reads the record in place.
struct DecodeLayout {
  uint32_t marks_off;  // mark bytes, a multiple of 32
  uint32_t mark_bytes;
  uint32_t flags_off;  // flag bytes of one record (+ 16 slack)
  uint32_t flag_bytes;
  uint32_t hi_off;     // k bytes (one-byte symbols, two-byte offsets) or none
  uint32_t io_off;     // output image + staged record
  uint32_t io_bytes;
  uint32_t per_warp;
  uint32_t staged;
};

// Largest record of a chunk of k symbols: flags, payload and (stream version
// 2, last chunk) up to S - 1 tail bytes.
__host__ __device__ inline uint64_t decode_record_bound(uint64_t k, uint32_t S, uint32_t offB,
                                                       uint32_t m) {
  const uint64_t extra = (1u + offB > S * m) ? (1u + offB - S * m) : 0u;
  return (k + 7) / 8 + static_cast<uint64_t>(S) * k + extra * (k / m) + (S - 1);
}

// Slack of the io area past the staged record (its end is at most this
// many bytes before the area's end, minus 15 for alignment).
constexpr uint32_t kIoSlack = 64;

// Slice for chunks of at most `kmax` symbols and `cmax` bytes whose records
// are at most `rmax` bytes; the full slice when `budget` bytes hold it,
// else without the io area.
__host__ __device__ inline DecodeLayout decode_layout(uint64_t kmax, uint64_t cmax,
                                                      uint64_t rmax, bool hi, bool shared,
                                                      uint64_t budget) {
  DecodeLayout L{};
  uint64_t at = 16;  // mbarrier
  L.marks_off = static_cast<uint32_t>(at);
  L.mark_bytes = static_cast<uint32_t>((kmax + 31) & ~31ull);
  at += L.mark_bytes;
  L.flags_off = static_cast<uint32_t>(at);
  L.flag_bytes = static_cast<uint32_t>(((kmax + 7) / 8 + 15) & ~15ull) + 16;
  at += L.flag_bytes;
  L.hi_off = static_cast<uint32_t>(at);
  if (hi) at += (kmax + 15) & ~15ull;
  const uint64_t base = at;
  L.io_off = static_cast<uint32_t>(at);
  const uint64_t c16 = ((cmax + 15) & ~15ull) + 16, r16 = (rmax + 15) & ~15ull;
  L.io_bytes = static_cast<uint32_t>((shared ? (c16 > r16 ? c16 : r16) : c16 + r16) + 32 +
                                     kIoSlack);
  at += L.io_bytes;
  L.staged = at <= budget;
  if (!L.staged) at = base;
  L.per_warp = static_cast<uint32_t>(at);
  return L;
}

struct DecompressBatchArgs {
  const DecItem *items;        // streams with at least one chunk
  const uint64_t *item_base;   // items[i].gbase, ascending
  uint32_t n_items;
  uint64_t total_chunks;
  const DecItem *empties;      // streams of zero bytes
  uint32_t n_empty;
  DecodeLayout lay;            // per-warp slice covering every stream
  uint32_t smem_bytes;         // dynamic shared memory per block
  uint32_t *err;
};

}  // namespace glz
