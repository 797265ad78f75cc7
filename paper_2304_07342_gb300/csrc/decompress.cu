// decompress.cu -- the decompression kernel (one warp per chunk).
//
// The paper only reports decompression throughput (section 4.4) and gives
// no algorithm; this is the design used here.  The host knows nothing
// about the stream: every warp reads and checks the header itself, so the
// call needs no host synchronisation.  Per chunk:
//   * the record offset is the superblock index entry plus the record sizes
//     of the (at most 63) chunks before it in its superblock -- no scan
//     across the whole stream;
//   * the record (flags + payload) is staged into the warp's shared slice
//     with a TMA bulk copy; a chunk without pointers (or a stored chunk of
//     stream version 2) is copied straight out with 16-byte stores;
//   * otherwise the chunk is decoded into a shared-memory image of its
//     output in two phases.  Phase 1 takes the tokens 32 at a time (lane =
//     token): the flag word gives each token's payload offset by popcount,
//     a shuffle scan of token lengths gives its output position; a literal
//     writes its symbol there, a pointer writes (offset - 1) into the slot
//     of its first symbol, and both mark their first position (one byte
//     per position: literal or pointer start).  Phase 2 takes the output
//     positions 32 at a time (lane = position): the owning token is the
//     last marked position at or before the position (a ballot and a bit
//     scan; a token that began in an earlier round is carried in
//     registers), a position
//     inside a pointer copies from position - offset, and sources inside
//     the same 32 positions are resolved by pointer jumping over the lanes;
//     earlier positions are final, later rounds read them;
//   * the image is copied out with 16-byte stores.
// Pointers never reach before their own chunk, so chunks are independent
// (section 3.3.1).  When the slice cannot hold the output image and the
// record window (very large chunks), the same two phases run on the output
// buffer itself and read the record in place.
#include <cuda_runtime.h>

#include "glz_common.h"
#include "glz_device.cuh"
#include "launch_cache.cuh"

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

// Worst-case record of a chunk of k symbols (flags + payload, no tail).
__device__ __forceinline__ uint64_t record_bound(uint64_t k, const Header &h) {
  const uint64_t extra = (1u + h.offB > h.S * h.m) ? (1u + h.offB - h.S * h.m) : 0u;
  return (k + 7) / 8 + static_cast<uint64_t>(h.S) * k + extra * (k / h.m);
}

// Little-endian 32-bit word at any byte address of shared memory (the two
// aligned words around it; may read up to 3 bytes past the addressed ones).
__device__ __forceinline__ uint32_t ld_u32_any(const uint8_t *p) {
  const uintptr_t a = reinterpret_cast<uintptr_t>(p);
  const uint32_t *w = reinterpret_cast<const uint32_t *>(a & ~static_cast<uintptr_t>(3));
  const uint32_t sh = 8u * static_cast<uint32_t>(a & 3u);
  return sh ? __funnelshift_r(w[0], w[1], sh) : w[0];
}

// Symbol slot j of an output image (S-byte aligned) or of an output buffer
// of any alignment.
template <int S>
__device__ __forceinline__ uint32_t ld_slot(const uint8_t *o, uint32_t j, bool aligned) {
  const uint8_t *p = o + static_cast<uint64_t>(j) * S;
  if constexpr (S == 1) return *p;
  if (aligned) {
    if constexpr (S == 2) return *reinterpret_cast<const uint16_t *>(p);
    else return *reinterpret_cast<const uint32_t *>(p);
  }
  return static_cast<uint32_t>(ld_le(p, S));
}

template <int S>
__device__ __forceinline__ void st_slot(uint8_t *o, uint32_t j, uint32_t v, bool aligned) {
  uint8_t *p = o + static_cast<uint64_t>(j) * S;
  if constexpr (S == 1) {
    *p = static_cast<uint8_t>(v);
    return;
  }
  if (aligned) {
    if constexpr (S == 2) *reinterpret_cast<uint16_t *>(p) = static_cast<uint16_t>(v);
    else *reinterpret_cast<uint32_t *>(p) = v;
    return;
  }
  for (uint32_t i = 0; i < S; ++i) p[i] = static_cast<uint8_t>(v >> (8 * i));
}

// Copy record bytes [src, src + n) to the end of the warp's io area (16-byte
// aligned, io_bytes long), ending at most kIoSlack bytes before it, so that
// the copy is 16-byte aligned on both sides: head and tail with plain
// loads, the middle with one TMA bulk copy.  Returns the shared address of
// byte 0.
__device__ __forceinline__ const uint8_t *stage_record(const uint8_t *src,
                                                       uint32_t n, uint8_t *io,
                                                       uint32_t io_bytes, uint64_t *bar,
                                                       uint32_t &phase,
                                                       uint32_t lane, bool &ok) {
  const uint32_t mis = static_cast<uint32_t>(reinterpret_cast<uintptr_t>(src) & 15u);
  uint8_t *dst = io + ((io_bytes - kIoSlack - n - 15) & ~15u) + mis;
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


// A warp's shared-memory slice (see DecodeLayout).
struct Slice {
  uint64_t *bar;
  uint8_t *marks;           // per position: 0 inside a token, 1 literal start, 2 pointer start
  uint8_t *hi;              // high bytes of (offset - 1), or nullptr
  uint8_t *fl;              // a copy of the record's flag bytes
  uint8_t *io;              // output image + staged record, or nullptr (decode
                            // into the output, read the record in place)
  uint32_t io_bytes, flag_bytes, mark_bytes;  // region sizes
  uint32_t phase;           // parity of the next TMA completion on bar
};

__device__ __forceinline__ Slice make_slice(uint8_t *ws, const DecodeLayout &L, bool hi) {
  Slice sl;
  sl.bar = reinterpret_cast<uint64_t *>(ws);
  sl.marks = ws + L.marks_off;
  sl.hi = hi ? ws + L.hi_off : nullptr;
  sl.fl = ws + L.flags_off;
  sl.io = L.staged ? ws + L.io_off : nullptr;
  sl.io_bytes = L.staged ? L.io_bytes : 0;
  sl.flag_bytes = L.flag_bytes;
  sl.mark_bytes = L.mark_bytes;
  sl.phase = 0;
  return sl;
}

// Flag word g of a record (tokens 32g .. 32g+31; bits of tokens past ntok
// cleared).  STAGED: the flags are in shared memory, where a word may be
// read past the flag bytes.
template <bool STAGED>
__device__ __forceinline__ uint32_t flag_word(const uint8_t *flags, uint32_t g, uint32_t ntok,
                                              uint32_t fb) {
  uint32_t fw;
  if constexpr (STAGED) {
    fw = ld_u32_any(flags + 4 * g);
  } else {
    fw = 0;
    for (uint32_t i = 0; i < 4; ++i)
      if (4 * g + i < fb) fw |= static_cast<uint32_t>(flags[4 * g + i]) << (8 * i);
  }
  const uint32_t left = ntok - 32 * g;
  return left >= 32 ? fw : fw & ((1u << left) - 1u);
}

// Phases 1 and 2 for a chunk of k symbols with ntok tokens whose payload
// holds pay_tok bytes of tokens: the symbols are written into `ob` (the
// output image, or the output itself).  STAGED: the record is in shared
// memory (words may be read up to 3 bytes past it).  False when the tokens
// are inconsistent (corrupt stream); nothing outside the chunk's output and
// the slice is written either way.
// SAME: a pointer's payload is S bytes like a literal's (1 + offB == S), so
// token t's payload starts at S * t without counting the pointers before it.
template <int S, bool STAGED, bool SAME = false>
__device__ __forceinline__ bool decode_tokens(const Header &h, const uint8_t *flags,
                                              const uint8_t *payload, uint32_t ntok,
                                              uint32_t pay_tok, uint32_t k, uint8_t *ob,
                                              bool aligned, const Slice &sl, uint32_t lane) {
  const uint32_t tsz = 1u + h.offB;
  const uint32_t offmask = h.offB == 2 ? 0xFFFFu : 0xFFu;
  const uint32_t lt = lanemask_lt(lane);
  const uint32_t fb = (ntok + 7) / 8;
  uint8_t *marks = sl.marks;
  {
    uint4 *m16 = reinterpret_cast<uint4 *>(marks);
    const uint32_t n16 = ((k + 31) & ~31u) / 16;
    for (uint32_t i = lane; i < n16; i += 32) m16[i] = make_uint4(0, 0, 0, 0);
  }
  __syncwarp();

  // Phase 1: tokens (lane = token), two groups of 32 per step.  The flag
  // words are read 32 at a time (lane = group); a scan of their popcounts
  // gives every group the pointers before it, so each token's payload
  // offset follows without a running sum: S bytes per literal and 1 + offB
  // per pointer before it.  The payload must hold exactly the flagged
  // tokens, checked before any token is read.
  const uint32_t ngroups = (ntok + 31) / 32;
  uint32_t np = 0;
  for (uint32_t g = lane; g < ngroups; g += 32)
    np += __popc(flag_word<STAGED>(flags, g, ntok, fb));
  np = __reduce_add_sync(kFull, np);
  if (S * (ntok - np) + tsz * np != pay_tok) return false;
  auto put = [&](uint32_t st, bool m, uint32_t off, uint32_t w) {
    if (!GLZ_OK(st < k && st < sl.mark_bytes)) return;
    marks[st] = m ? 2 : 1;
    st_slot<S>(ob, st, m ? off - 1u : w, aligned);
    if (S == 1 && sl.hi && m) sl.hi[st] = static_cast<uint8_t>((off - 1u) >> 8);
  };
  uint32_t pos = 0, pdone = 0;  // symbols produced; pointers in earlier blocks of groups
  for (uint32_t g0 = 0; g0 < ngroups; g0 += 32) {
    const uint32_t fwr = g0 + lane < ngroups ? flag_word<STAGED>(flags, g0 + lane, ntok, fb) : 0u;
    uint32_t pb = 0;  // pointers before group g0 + lane (not needed when SAME)
    if constexpr (!SAME) {
      const uint32_t cnt = __popc(fwr);
      uint32_t incl = cnt;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(kFull, incl, o);
        if (lane >= static_cast<uint32_t>(o)) incl += y;
      }
      pb = pdone + incl - cnt;
      pdone += __shfl_sync(kFull, incl, 31);
    }
    const uint32_t nblk = min(32u, ngroups - g0);
    for (uint32_t i = 0; i < nblk; i += 2) {
      const bool hasB = i + 1 < nblk;
      const uint32_t fwA = __shfl_sync(kFull, fwr, i);
      const uint32_t fwB = __shfl_sync(kFull, fwr, (i + 1) & 31u);
      const uint32_t tA = (g0 + i) * 32 + lane, tB = tA + 32;
      const bool vA = tA < ntok, vB = hasB && tB < ntok;
      const bool mA = (fwA >> lane) & 1u, mB = hasB && ((fwB >> lane) & 1u);
      uint32_t oA = S * tA, oB = S * tB;
      if constexpr (!SAME) {
        const uint32_t pbA = __shfl_sync(kFull, pb, i), pbB = __shfl_sync(kFull, pb, (i + 1) & 31u);
        const uint32_t nbA = pbA + __popc(fwA & lt), nbB = pbB + __popc(fwB & lt);
        oA = S * (tA - nbA) + tsz * nbA;
        oB = S * (tB - nbB) + tsz * nbB;
      }
      uint32_t wA = 0, wB = 0;
      if constexpr (STAGED) {
        if (vA && GLZ_OK(oA < pay_tok)) wA = ld_u32_any(payload + oA);
        if (vB && GLZ_OK(oB < pay_tok)) wB = ld_u32_any(payload + oB);
      } else {
        if (vA) wA = static_cast<uint32_t>(ld_le(payload + oA, mA ? tsz : S));
        if (vB) wB = static_cast<uint32_t>(ld_le(payload + oB, mB ? tsz : S));
      }
      const uint32_t lenA = mA ? (wA & 0xFFu) : (vA ? 1u : 0u);
      const uint32_t lenB = mB ? (wB & 0xFFu) : (vB ? 1u : 0u);
      const uint32_t offA = mA ? ((wA >> 8) & offmask) + 1u : 0u;
      const uint32_t offB = mB ? ((wB >> 8) & offmask) + 1u : 0u;
      // inclusive scans of both groups' token lengths in one: A in the low
      // and B in the high 16 bits (a group's lengths sum to at most
      // 32 x 255, so the halves never carry into each other)
      uint32_t x = lenA | (lenB << 16);
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(kFull, x, o);
        if (lane >= static_cast<uint32_t>(o)) x += y;
      }
      const uint32_t gl2 = __shfl_sync(kFull, x, 31);
      const uint32_t xA = x & 0xFFFFu, xB = x >> 16;
      const uint32_t glA = gl2 & 0xFFFFu, glB = gl2 >> 16;
      const uint32_t sA = pos + xA - lenA, sB = pos + glA + xB - lenB;
      // a pointer needs 1 <= length <= offset (any length <= 255 in overlap
      // mode) and offset <= min(W, its start): its source lies in the chunk
      const uint32_t capA = h.overlap ? 256u : offA, capB = h.overlap ? 256u : offB;
      const bool bad = (mA && !(lenA - 1u < capA && offA <= min(h.W, sA))) ||
                       (mB && !(lenB - 1u < capB && offB <= min(h.W, sB)));
      if (__any_sync(kFull, bad) || pos + glA + glB > k) return false;
      pos += glA + glB;
      if (vA) put(sA, mA, offA, wA);
      if (vB) put(sB, mB, offB, wB);
    }
  }
  if (pos != k) return false;
  __syncwarp();

  // Phase 2: positions, 32 at a time (lane = position)
  const uint32_t le = lt | (1u << lane);
  uint32_t carry = 0;  // offset of the pointer owning the previous round's last position (0: literal)
  for (uint32_t r0 = 0; r0 < k; r0 += 32) {
    const uint32_t j = r0 + lane;
    const bool act = j < k;
    const uint32_t mk = marks[j];  // zero past k
    const uint32_t sw = __ballot_sync(kFull, mk != 0);
    // the offset of the pointer starting here (its slot holds offset - 1);
    // 0 at a literal's start
    uint32_t so = 0;
    if constexpr (S == 1) {  // (a byte load costs less than the branch around it)
      uint32_t raw = act ? ld_slot<S>(ob, j, aligned) : 0u;
      if (sl.hi && act) raw |= static_cast<uint32_t>(sl.hi[j]) << 8;
      so = mk == 2 ? raw + 1u : 0u;
    } else if (mk == 2) {
      so = ld_slot<S>(ob, j, aligned) + 1u;
    }
    const uint32_t mb = sw & le;
    const uint32_t ol = (31u - __clz(mb)) & 31u;  // owner's lane when mb != 0
    const uint32_t oso = __shfl_sync(kFull, so, ol);
    const uint32_t own = mb ? oso : carry;
    carry = __shfl_sync(kFull, own, 31);
    const bool ptr = act && own != 0;
    uint32_t f = ptr ? j - own : j;
    // sources inside this round that are pointer symbols themselves are not
    // final yet: jump (f <- the source's source, all lanes at once) until
    // every source is a literal of the round or lies before it (chains
    // shrink, so at most 5 turns)
    const uint32_t pm = __ballot_sync(kFull, ptr);
    auto pending = [&](uint32_t x) { return x >= r0 && ((pm >> (x - r0)) & 1u); };
    while (__any_sync(kFull, pending(f))) f = __shfl_sync(kFull, f, pending(f) ? f - r0 : lane);
    if (ptr && GLZ_OK(f < j)) st_slot<S>(ob, j, ld_slot<S>(ob, f, aligned), aligned);
    __syncwarp();
  }
  return true;
}

template <bool STAGED>
__device__ __forceinline__ bool decode_tokens_s(const Header &h, const uint8_t *flags,
                                                const uint8_t *payload, uint32_t ntok,
                                                uint32_t pay_tok, uint32_t k, uint8_t *ob,
                                                bool aligned, const Slice &sl, uint32_t lane) {
  switch (h.S) {
    case 1:
      return decode_tokens<1, STAGED>(h, flags, payload, ntok, pay_tok, k, ob, aligned, sl, lane);
    case 2:
      if (h.offB == 1)  // a pointer (length, offset - 1) is two bytes, as a symbol
        return decode_tokens<2, STAGED, true>(h, flags, payload, ntok, pay_tok, k, ob, aligned, sl,
                                              lane);
      return decode_tokens<2, STAGED>(h, flags, payload, ntok, pay_tok, k, ob, aligned, sl, lane);
    default:
      return decode_tokens<4, STAGED>(h, flags, payload, ntok, pay_tok, k, ob, aligned, sl, lane);
  }
}

// One chunk.  Returns false when a TMA copy did not complete in time (the
// warp must stop: its barrier phase is unknown).
__device__ __forceinline__ bool decode_chunk(const DecompressArgs &A, const Header &h,
                                             uint32_t c, uint64_t records_at, Slice &sl,
                                             uint32_t lane) {
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
  const uint8_t *flags = in + rec_at;  // read in place when there is no io area
  if (sl.io) {
    bool staged;
    if (!GLZ_OK(fb + pay + kIoSlack + 15 <= sl.io_bytes)) return true;
    flags = stage_record(in + rec_at, static_cast<uint32_t>(fb + pay), sl.io, sl.io_bytes,
                         sl.bar, sl.phase, lane, staged);
    if (!staged) {
      if (lane == 0) atomicOr(A.err, kErrTimeout);
      return false;
    }
  }
  const uint8_t *payload = flags + fb;
  uint8_t *dst = A.out + chunk_at;
  if (stored) {
    if (sl.io) {
      copy_s2g(dst, payload, pay, lane);  // the io area has slack past the record
    } else {
      for (uint32_t i = lane; i < pay; i += 32) dst[i] = payload[i];
    }
    return true;
  }
  // a chunk without pointers is its payload: copy it straight out
  uint32_t any = 0;
  for (uint32_t i = lane; i < fb; i += 32) any |= flags[i];
  if (!__any_sync(kFull, any != 0)) {
    if (ntok != k || pay != bytes_c) {
      if (lane == 0) atomicOr(A.err, kErrCorrupt);
      return true;
    }
    if (sl.io) {
      copy_s2g(dst, payload, pay, lane);
    } else {
      for (uint32_t i = lane; i < pay; i += 32) dst[i] = payload[i];
    }
    return true;
  }
  const uint32_t pay_tok = pay - tail;  // the tokens' payload; the tail follows it
  // the tail bytes, read before the output image may grow over the record
  const uint8_t tb = lane < tail ? payload[pay_tok + lane] : 0;
  bool ok;
  if (sl.io) {
    // the flag bytes are copied out first: the output image grows from the
    // start of the io area towards the record's flags
    if (!GLZ_OK(fb + 8 <= sl.flag_bytes)) return true;
    for (uint32_t i = lane; i < fb; i += 32) sl.fl[i] = flags[i];
    __syncwarp();
    ok = decode_tokens_s<true>(h, sl.fl, payload, ntok, pay_tok, k, sl.io, true, sl, lane);
  } else {
    const bool aligned = A.out_aligned != 0 && (h.C % 4) == 0;
    ok = decode_tokens_s<false>(h, flags, payload, ntok, pay_tok, k, dst, aligned, sl, lane);
  }
  if (!ok) {
    if (lane == 0) atomicOr(A.err, kErrCorrupt);
    return true;
  }
  uint8_t *ob = sl.io ? sl.io : dst;
  if (lane < tail) ob[static_cast<uint64_t>(k) * h.S + lane] = tb;
  if (sl.io && GLZ_OK(bytes_c + 16 <= sl.io_bytes && chunk_at + bytes_c <= A.out_cap)) {
    __syncwarp();
    copy_s2g(dst, sl.io, bytes_c, lane);
  }
  __syncwarp();
  return true;
}

// Per-warp slice for a stream with header h.
__device__ __forceinline__ DecodeLayout layout_of(const Header &h, uint64_t budget) {
  const uint64_t k = h.C / h.S;
  return decode_layout(k, h.C, decode_record_bound(k, h.S, h.offB, h.m), h.S == 1 && h.offB == 2,
                       h.S * h.m >= 1 + h.offB, budget);
}

}  // namespace

__global__ void __launch_bounds__(1024, 1) decompress_kernel(const DecompressArgs A) {
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
  // per-warp slice, decided from the header; warps that do not fit sit out
  const DecodeLayout L = layout_of(h, A.smem_bytes);
  const uint32_t fit = A.smem_bytes / L.per_warp;
  const uint32_t active = fit < wpb ? fit : wpb;
  if (warp >= active) return;
  Slice sl = make_slice(smem + static_cast<uint64_t>(warp) * L.per_warp, L,
                        h.S == 1 && h.offB == 2);
  if (lane == 0) {
    mbar_init(sl.bar, 1);
    fence_mbar_init();
  }
  __syncwarp();
  const uint32_t gw = blockIdx.x * active + warp;
  const uint32_t nwarps = gridDim.x * active;
  for (uint32_t c = gw; c < h.nc; c += nwarps)
    if (!decode_chunk(A, h, c, records_at, sl, lane)) break;
  if (lane == 0) checked_fold(A.err);
}

// Batched decompression: chunks of all streams in order, grid-stride; each
// warp finds its stream by a 32-way search over the streams' first chunks.
__global__ void __launch_bounds__(1024, 1) decompress_batch_kernel(const DecompressBatchArgs B) {
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
  const uint32_t fit = B.smem_bytes / B.lay.per_warp;
  const uint32_t active = fit < wpb ? fit : wpb;
  if (warp >= active) return;
  // the slice covers every stream; the high-byte area exists when any needs it
  Slice base = make_slice(smem + static_cast<uint64_t>(warp) * B.lay.per_warp, B.lay, false);
  if (lane == 0) {
    mbar_init(base.bar, 1);
    fence_mbar_init();
  }
  __syncwarp();
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
    // the header must still be the one the plan sized the slices for
    const uint64_t kh = ok ? h.C / h.S : 0;
    const bool need_hi = ok && h.S == 1 && h.offB == 2;
    // the io area: a stream whose pointers may outgrow their symbols needs
    // the output image and the record side by side
    auto fits_io = [](const DecodeLayout &L, const Header &hh, uint64_t kk) {
      const uint64_t c16 = ((hh.C + 15) & ~15ull) + 16;
      const uint64_t r16 = (decode_record_bound(kk, hh.S, hh.offB, hh.m) + 15) & ~15ull;
      const bool sh = hh.S * hh.m >= 1 + hh.offB;
      return (sh ? (c16 > r16 ? c16 : r16) : c16 + r16) + 32 + kIoSlack <= L.io_bytes;
    };
    const bool fits = ok && h.nc == it.nc && kh <= B.lay.mark_bytes &&
                      (!need_hi || B.lay.io_off - B.lay.hi_off >= kh) &&
                      (kh + 7) / 8 + 8 <= B.lay.flag_bytes &&
                      (!B.lay.staged || fits_io(B.lay, h, kh)) &&
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
    base.hi = need_hi ? smem + static_cast<uint64_t>(warp) * B.lay.per_warp + B.lay.hi_off
                      : nullptr;
    if (!decode_chunk(A, h, c, records_at, base, lane)) break;
  }
  if (lane == 0) checked_fold(B.err);
}

cudaError_t launch_decompress_batch(DecompressBatchArgs B, int block, cudaStream_t stream) {
  static LaunchCache lc;
  const size_t smem = B.smem_bytes;
  int per_sm = 0, sms = 0;
  cudaError_t e = resident_blocks(lc, decompress_batch_kernel, block, smem, &per_sm, &sms);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  const uint64_t warps = block / 32;
  uint64_t want = (B.total_chunks + warps - 1) / warps;
  if (want == 0) want = 1;
  const uint64_t cap = static_cast<uint64_t>(per_sm) * sms;
  const unsigned grid = static_cast<unsigned>(want < cap ? want : cap);
  decompress_batch_kernel<<<grid, block, smem, stream>>>(B);
  return cudaGetLastError();
}

cudaError_t launch_decompress(DecompressArgs A, int block, cudaStream_t stream) {
  static LaunchCache lc;
  const size_t smem = A.smem_bytes;
  int per_sm = 0, sms = 0;
  cudaError_t e = resident_blocks(lc, decompress_kernel, block, smem, &per_sm, &sms);
  if (e != cudaSuccess) return e;
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
