// compress_impl.cuh -- the fused compression kernel (one warp per chunk).
//
// gpuLZ splits compression into Kernel I (match + local prefix sum +
// encode, section 3.3.2), Kernel II (global prefix sum, 3.3.3) and Kernel
// III (deflate, 3.3.4).  Here all of it is one persistent kernel; each warp
// takes the next chunk from a work counter and
//   1. stages the chunk into its shared-memory slice (1-D TMA bulk copy);
//   2. checks whether any position can start a match at all (a Bloom
//      filter over symbol keys, tried after a chunk without pointers;
//      chunks without repeats end here as all literals), else links every
//      position to the last earlier position with the same hash of its
//      first min(m, 8/S) symbols (hash chains; __match_any_sync links
//      positions of one 32-position slab) and marks the positions whose
//      chain holds their key inside the window -- only those can start a
//      match of >= m symbols;
//   3. walks the greedy parse (section 2.2 steps 1-6): the next 32 marked
//      positions are evaluated in parallel, one lane each, by walking their
//      chains nearest-first and extending every candidate exactly (length
//      <= offset, section 3.3.2; not bounded by the offset in the overlap
//      mode of stream version 2) or, with the paper's matcher, by the
//      paper's forward scan of the window.  The parse through the batch is
//      found by a short chase over lanes, then warp scans give each token
//      its index and payload offset (the local, first pass of the two-pass
//      prefix sum of section 3.2.2) and the lanes write the tokens in
//      parallel into a staging record in shared memory;
//   4. in stream version 2, appends the bytes after the last whole symbol
//      and stores the chunk as it is if its record would not be smaller;
//   5. obtains its record's global offset from a decoupled look-back over
//      the chunks before it (the second pass) -- bounded spins, no extra
//      kernel, no per-symbol data in HBM -- or parks the record (by
//      reference when it is the chunk's own input) and moves on;
//   6. writes its table entry, index entry and record at the final offset.
#pragma once

#include <cstdint>

#include "glz_common.h"
#include "glz_device.cuh"

namespace glz {

template <int S>
struct SymType;
template <>
struct SymType<1> {
  using T = uint8_t;
};
template <>
struct SymType<2> {
  using T = uint16_t;
};
template <>
struct SymType<4> {
  using T = uint32_t;
};

constexpr uint16_t kNoPos = 0xFFFF;  // chunk positions are < 32768

// Chain links: distance from a position to the previous one with the same
// key hash.  One byte per position while W <= 256 (two bytes beyond),
// holding distance - 1; a position without a link within the window holds
// all ones, read as distance 256 (or 65536).  A walk only starts at a
// position that has a link (a marked one), and after its first hop any step
// of 256 or more leaves the window (W <= 256 for one-byte links), so the
// sentinel and a true link of 256 both end the walk where they should.
template <bool WIDE>
struct Links {
  uint8_t *base;
  __device__ __forceinline__ uint32_t get(uint32_t p) const {
    if constexpr (WIDE) return 1u + reinterpret_cast<const uint16_t *>(base)[p];
    else return 1u + base[p];
  }
  __device__ __forceinline__ void set(uint32_t p, uint32_t d) const {  // 0: none
    if constexpr (WIDE)
      reinterpret_cast<uint16_t *>(base)[p] = static_cast<uint16_t>(d - 1);
    else
      base[p] = static_cast<uint8_t>(d - 1);
  }
};

// Little-endian 32-bit word of the chunk starting at byte b (any alignment;
// reads the aligned words around it).
__device__ __forceinline__ uint32_t bytes_at(const uint8_t *base, uint32_t b) {
  const uint32_t *w = reinterpret_cast<const uint32_t *>(base + (b & ~3u));
  const uint32_t sh = 8u * (b & 3u);
  return sh ? __funnelshift_r(w[0], w[1], sh) : w[0];
}

// Key of position p: its first g symbols, S * g <= 8 little-endian bytes,
// as two 32-bit words (the bytes beyond the key masked off).
template <int S>
__device__ __forceinline__ void key_at(const uint8_t *in, uint32_t p, uint32_t mlo,
                                       uint32_t mhi, uint32_t &lo, uint32_t &hi) {
  lo = bytes_at(in, p * S) & mlo;
  hi = mhi ? bytes_at(in, p * S + 4) & mhi : 0u;
}

// Step 2: hash chains.  For every position p with room for m symbols, the
// key is its first g = min(m, 8/S) symbols; the link of p is the distance to
// the last earlier position with the same key hash when that lies within
// the window.  A match of >= m symbols at p from offset d needs p - d to
// carry the same key, so every such offset is on p's chain.
// Bit p of `maybe` marks the positions whose chain can hold such an offset:
// one of the first kFilterHops entries of p's chain within the window
// carries p's key, or the chain goes on within the window beyond them.
// Unmarked positions have no offset with p's key in the window, so skipping
// them as literals leaves the greedy parse unchanged; the test drops the
// positions that only share a hash (nearly all of them on data without
// repeats, whose chunks then skip the parse altogether).
//
// The table holds the last position of each hash.  Slabs of 32 positions
// go through it in order: each lane reads its bucket, then all lanes write
// their position and read it back; a lane that finds another position lost
// a collision, so its slab holds two positions with one hash.  Only such
// slabs need the lane groups of __match_any_sync (a shared unit with low
// throughput).  The key filter runs after kGroup slabs have been linked, on
// independent loads.
constexpr uint32_t kFilterHops = 1;  // chain entries the candidate filter inspects

template <int S, bool WIDE>
__device__ __forceinline__ void build_chains(const typename SymType<S>::T *sym,
                                             uint32_t k, const BufDesc &A,
                                             const CompressSmem &sm, uint16_t *table,
                                             uint32_t *maybe, const Links<WIDE> &links,
                                             uint32_t lane) {
  const uint32_t H = 1u << sm.hash_log2;  // >= 16
  uint4 *t4 = reinterpret_cast<uint4 *>(table);
  for (uint32_t i = lane; i < H / 8; i += 32) t4[i] = make_uint4(kFull, kFull, kFull, kFull);
  __syncwarp();

  const uint8_t *in = reinterpret_cast<const uint8_t *>(sym);
  const uint32_t kb = S * min(A.m, 8u / S);  // key bytes
  const uint32_t mlo = kb >= 4 ? kFull : (1u << (8 * kb)) - 1u;
  const uint32_t mhi = kb <= 4 ? 0u : (kb >= 8 ? kFull : (1u << (8 * (kb - 4))) - 1u);
  const uint32_t tshift = 32u - sm.hash_log2;
  const uint32_t lt = lanemask_lt(lane);
  const uint32_t nslab = (k + 31) / 32;
  constexpr uint32_t kGroup = 2;  // slabs whose hashes and filters are formed together
  for (uint32_t s0 = 0; s0 < nslab; s0 += kGroup) {
    uint32_t hh[kGroup], klo[kGroup], khi[kGroup], qq[kGroup], dd[kGroup];
    bool okk[kGroup];
#pragma unroll
    for (uint32_t u = 0; u < kGroup; ++u) {
      const uint32_t p = (s0 + u) * 32 + lane;
      const bool ok = s0 + u < nslab && p + A.m <= k;  // room for m symbols
      uint32_t lo = 0, hi = 0;
      if (ok) key_at<S>(in, p, mlo, mhi, lo, hi);
      hh[u] = ((hi * 0x85EBCA77u ^ lo) * 0x9E3779B1u) >> tshift;
      klo[u] = lo;
      khi[u] = hi;
      okk[u] = ok;
    }
    // links, slab after slab
#pragma unroll
    for (uint32_t u = 0; u < kGroup; ++u) {
      qq[u] = kNoPos;
      dd[u] = 0;
      if (s0 + u >= nslab) continue;
      const uint32_t base = (s0 + u) * 32;
      const uint32_t p = base + lane;
      const bool ok = okk[u];
      const uint32_t h = hh[u];
      const bool hok = GLZ_OK(h < H);
      const uint32_t old = ok && hok ? table[h] : kNoPos;
      __syncwarp();
      if (ok && hok) table[h] = static_cast<uint16_t>(p);
      __syncwarp();
      const bool lost = ok && hok && table[h] != p;
      uint32_t q = old;
      if (__any_sync(kFull, lost)) {
        const uint32_t grp = __match_any_sync(kFull, ok ? h : (0x10000u + lane));
        const uint32_t lower = grp & lt;
        if (lower) q = base + (31u - __clz(lower));
        __syncwarp();
        if (ok && hok && (grp >> lane) == 1u) table[h] = static_cast<uint16_t>(p);  // last wins
      }
      const uint32_t dist = (ok && q != kNoPos && p - q <= A.W) ? p - q : 0u;
      if (p < k && GLZ_OK(dist <= p)) links.set(p, dist);
      qq[u] = q;
      dd[u] = dist;
    }
    __syncwarp();
    // candidate filter: walk p's chain for a position with p's key while it
    // stays in the window (a few hops; past them p stays marked)
#pragma unroll
    for (uint32_t u = 0; u < kGroup; ++u) {
      uint32_t cur = qq[u], reach = dd[u];
      bool mb = false;
      if (reach) {
        for (uint32_t hop = 0;; ++hop) {
          uint32_t lo, hi;
          key_at<S>(in, cur, mlo, mhi, lo, hi);
          if (lo == klo[u] && hi == khi[u]) {
            mb = true;
            break;
          }
          const uint32_t step = links.get(cur);  // >= 256 when none (see Links)
          if (reach + step > A.W) break;
          if (hop + 1 == kFilterHops) {
            mb = true;
            break;
          }
          cur -= step;
          reach += step;
        }
      }
      const uint32_t mbits = __ballot_sync(kFull, mb);
      if (lane == 0 && s0 + u < nslab && GLZ_OK(s0 + u < (sm.mbar_off - sm.maybe_off) / 4))
        maybe[s0 + u] = mbits;
    }
    __syncwarp();
  }
}

// Literal pre-check: true only when no position of the chunk can start a
// match of >= m symbols, so that the greedy parse is k literals (section
// 2.2: a position without a match is emitted as a literal) and the chains
// need not be built.  It is exact in both directions that matter: it never
// returns true for a chunk with a match, and on data without repeats it
// returns true after one shared-memory atomic per position.
//
// Every position with room for m symbols ORs a 4-bit mask, drawn from a hash
// of its key (its first g symbols, as for the chains), into one 32-bit word
// of a bitmap that starts empty (a blocked Bloom filter over the keys seen
// so far in the chunk; the word is the high half of hash x word count, so
// the bitmap fills whatever shared memory the chains would use, about 10
// bits per position for 4-byte symbols).  The atomic returns the word before
// the OR; a
// position finds all its bits already set ("flagged") whenever an earlier
// position of an earlier slab has its key.  Two positions of one slab that
// share a key are ordered by the atomic unit, not by position, so it is the
// one processed second that is flagged, which may be the earlier position.
// So a flagged position p is checked exactly, by the whole warp, for
//   (i)  a match of >= m symbols at p from an offset d in [m, min(W, p)], and
//   (ii) a match of >= m symbols at a later position of p's own slab from p;
// and any hit (or more than kBloomMaxFlagged flagged positions) sends the
// chunk to the full path.  If some position q has a match from p = q - d,
// then p and q share the key: q is flagged (and (i) finds it) unless p and q
// lie in one slab and p came second, in which case p is flagged and (ii)
// finds it.
constexpr uint32_t kBloomMaxFlagged = 16;
constexpr uint32_t kBloomGroup = 8;  // slabs whose ORs are issued together

// Does p (flagged, p + m <= k) take part in a match of >= m symbols, as the
// position coded ((i)) or as the source of a later position of its slab
// that ends at `slab_end` ((ii))?  Warp-wide; every lane returns the answer.
// (i) takes four offsets per lane per round: their first symbols are loaded
// before any is compared, so the loads overlap.
template <int S>
__device__ __forceinline__ bool match_near(const typename SymType<S>::T *sym, uint32_t k,
                                           const BufDesc &A, uint32_t p, uint32_t slab_end,
                                           uint32_t lane) {
  using Sym = typename SymType<S>::T;
  const uint32_t dmax = min(A.W, p);
  // a match of >= m symbols needs offset >= m unless matches may overlap
  const uint32_t dmin = A.match == kMatchOverlap ? 1u : A.m;
  const Sym first = sym[p];
  bool hit = false;
  for (uint32_t d0 = 0; d0 < dmax; d0 += 128) {
    Sym v[4];
#pragma unroll
    for (uint32_t u = 0; u < 4; ++u) {
      const uint32_t d = d0 + 32 * u + lane + 1;
      v[u] = d <= dmax ? sym[p - d] : first;
    }
#pragma unroll
    for (uint32_t u = 0; u < 4; ++u) {
      const uint32_t d = d0 + 32 * u + lane + 1;
      bool eq = v[u] == first && d >= dmin && d <= dmax;
      for (uint32_t i = 1; eq && i < A.m; ++i) eq = sym[p + i] == sym[p - d + i];
      hit |= eq;
    }
  }
  const uint32_t q = p + 1 + lane;
  bool eq = q < slab_end && (q - p >= A.m || A.match == kMatchOverlap) && q - p <= A.W &&
            q + A.m <= k;
  for (uint32_t i = 0; eq && i < A.m; ++i) eq = sym[q + i] == sym[p + i];
  hit |= eq;
  return __any_sync(kFull, hit);
}

// `bm` holds `nwords` words (a multiple of 4, 16-byte aligned).
template <int S>
__device__ __forceinline__ bool literal_chunk(const typename SymType<S>::T *sym, uint32_t k,
                                              const BufDesc &A, uint32_t *bm, uint32_t nwords,
                                              uint32_t *maybe, uint32_t lane) {
  uint4 *b4 = reinterpret_cast<uint4 *>(bm);
  for (uint32_t i = lane; i < nwords / 4; i += 32) b4[i] = make_uint4(0, 0, 0, 0);
  __syncwarp();
  const uint8_t *in = reinterpret_cast<const uint8_t *>(sym);
  const uint32_t kb = S * min(A.m, 8u / S);  // key bytes, as in build_chains
  const uint32_t mlo = kb >= 4 ? kFull : (1u << (8 * kb)) - 1u;
  const uint32_t mhi = kb <= 4 ? 0u : (kb >= 8 ? kFull : (1u << (8 * (kb - 4))) - 1u);
  const uint32_t nslab = (k + 31) / 32;
  uint32_t nflag = 0;
  // groups of kBloomGroup slabs: keys and masks first, then the ORs in slab
  // order (each behind the previous one), then the votes, so that the ORs of
  // a group are in flight together
  for (uint32_t s0 = 0; s0 < nslab; s0 += kBloomGroup) {
    uint32_t widx[kBloomGroup], mask[kBloomGroup], old[kBloomGroup];
    bool okk[kBloomGroup];
#pragma unroll
    for (uint32_t u = 0; u < kBloomGroup; ++u) {
      const uint32_t p = (s0 + u) * 32 + lane;
      const bool ok = s0 + u < nslab && p + A.m <= k;
      uint32_t lo = 0, hi = 0;
      if (ok) key_at<S>(in, p, mlo, mhi, lo, hi);
      const uint32_t h = ((hi * 0x85EBCA77u) ^ lo) * 0x9E3779B1u;
      const uint32_t g = h * 0xC2B2AE3Du;
      widx[u] = __umulhi(h, nwords);
      mask[u] = (1u << (g >> 27)) | (1u << ((g >> 22) & 31u)) | (1u << ((g >> 17) & 31u)) |
                (1u << ((g >> 12) & 31u));
      okk[u] = ok;
    }
#pragma unroll
    for (uint32_t u = 0; u < kBloomGroup; ++u) {
      old[u] = okk[u] && GLZ_OK(widx[u] < nwords) ? atomicOr(&bm[widx[u]], mask[u]) : 0u;
      __syncwarp();  // slab u's ORs before slab u+1's
    }
#pragma unroll
    for (uint32_t u = 0; u < kBloomGroup; ++u) {
      const uint32_t f = __ballot_sync(kFull, okk[u] && (old[u] & mask[u]) == mask[u]);
      if (lane == 0 && s0 + u < nslab) maybe[s0 + u] = f;
      nflag += __popc(f);
    }
    if (nflag > kBloomMaxFlagged) return false;
  }
  __syncwarp();
  if (nflag == 0) return true;
  for (uint32_t w0 = 0; w0 < nslab; w0 += 32) {
    const uint32_t f = w0 + lane < nslab ? maybe[w0 + lane] : 0u;
    uint32_t has = __ballot_sync(kFull, f != 0);
    while (has) {
      const uint32_t j = __ffs(has) - 1;
      has &= has - 1;
      uint32_t bits = __shfl_sync(kFull, f, j);
      const uint32_t s = w0 + j;
      while (bits) {
        const uint32_t p = s * 32 + __ffs(bits) - 1;
        bits &= bits - 1;
        if (match_near<S>(sym, k, A, p, min(k, s * 32 + 32), lane)) return false;
      }
    }
  }
  return true;
}

__device__ __forceinline__ void warp_copy_bytes(uint8_t *dst, const uint8_t *src,
                                                uint32_t nbytes, uint32_t lane) {
  warp_copy(dst, src, nbytes, lane);
}

// Length of the match at p from offset d (d >= 1), at most `cap` symbols.
template <int S>
__device__ __forceinline__ uint32_t extend(const typename SymType<S>::T *sym,
                                           uint32_t p, uint32_t d, uint32_t cap) {
  uint32_t l = 0;
  while (l < cap && sym[p + l] == sym[p - d + l]) ++l;
  return l;
}

// extend() four bytes at a time: compare 32-bit words of the look-ahead and
// of the source, and locate the first differing symbol with a bit scan.
// Reads up to 3 bytes beyond the compared symbols (within the staged chunk
// region and its slack).
template <int S>
__device__ __forceinline__ uint32_t extend_words(const uint8_t *in, uint32_t p,
                                                 uint32_t d, uint32_t cap) {
  constexpr uint32_t per = 4 / S;  // symbols per word
  uint32_t l = 0;
  if (!GLZ_OK(d <= p)) return 0;
  while (l < cap) {
    const uint32_t x = bytes_at(in, (p + l) * S) ^ bytes_at(in, (p - d + l) * S);
    if (x) return min(cap, l + static_cast<uint32_t>(__ffs(x) - 1) / (8 * S));
    l += per;
  }
  return cap;
}

// Per-lane work caps of the chain evaluation; a position that needs more
// (long repetitive runs) is left to the exact window walk below.
constexpr uint32_t kChainHops = 48;
constexpr uint32_t kChainWork = 384;

// Exact longest match at position q (one lane): walk q's chain, nearest
// offset first, extending every offset d >= m that could still beat the
// best; a strictly longer match replaces the best, so ties keep the nearest.
// Returns false when the work cap stopped the walk with candidates left.
template <int S, bool WIDE>
__device__ __forceinline__ bool chain_match(const typename SymType<S>::T *sym,
                                            uint32_t k, const BufDesc &A,
                                            const Links<WIDE> &links, uint32_t q,
                                            uint32_t &best, uint32_t &bd) {
  const bool overlap = A.match == kMatchOverlap;  // lengths not bounded by the offset
  const uint32_t lim = min(A.M, k - q);
  best = 0;
  bd = 0;
  uint32_t d = links.get(q), hops = 0, work = 0;
  while (d <= A.W) {
    if (best == lim) return true;
    if (hops >= kChainHops || work >= kChainWork) return false;
    // the next link is loaded first, so that its latency overlaps the
    // evaluation of this candidate (a link is >= 1; past the chain's end it
    // reads as a distance that leaves the window)
    const uint32_t step = GLZ_OK(d <= q) ? links.get(q - d) : 0x10000u;
    if (overlap || d >= A.m) {
      const uint32_t cap = overlap ? lim : min(lim, d);
      // only a candidate that agrees at index `best` can be longer
      if (cap > best && sym[q + best] == sym[q - d + best]) {
        const uint32_t l = extend_words<S>(reinterpret_cast<const uint8_t *>(sym), q, d, cap);
        work += l / (4 / S) + 1;
        if (l > best) {
          best = l;
          bd = d;
        }
      }
    }
    ++hops;
    d += step;
  }
  return true;
}

// First position w' in [w, p) with sym[w'] == c, or p if there is none.
// One aligned 32-bit word (4/S symbols) per step for S < 4.
template <int S>
__device__ __forceinline__ uint32_t next_equal(const typename SymType<S>::T *sym, uint32_t w,
                                               uint32_t p, typename SymType<S>::T c) {
  if constexpr (S == 4) {
    while (w < p && sym[w] != c) ++w;
    return w;
  } else {
    constexpr uint32_t per = 4 / S;
    const uint32_t *w32 = reinterpret_cast<const uint32_t *>(sym);
    const uint32_t rep = S == 1 ? 0x01010101u * c : 0x00010001u * c;
    while (w < p) {
      const uint32_t first = w & ~(per - 1);  // first symbol of w's word
      uint32_t eq = S == 1 ? __vcmpeq4(w32[first / per], rep) : __vcmpeq2(w32[first / per], rep);
      eq &= kFull << (8u * S * (w - first));  // symbols before w do not count
      if (eq) return min(p, first + static_cast<uint32_t>(__ffs(eq) - 1) / (8u * S));
      w = first + per;
    }
    return p;
  }
}

// The paper's matcher at position p (section 3.3.2, the four steps of its
// matching method), one lane per position.  The search pointer starts at
// the window start; at a symbol equal to the one at p a run starts and both
// pointers advance while the symbols agree; at a mismatch the run is kept
// if strictly longer than the best, the position pointer returns to p and
// the search pointer moves on from the symbol that broke the run (it never
// goes back).  The scan ends when a run reaches p (length <= offset) or the
// end of the look-ahead (the chunk end or M symbols, whichever is first).
// Here the search pointer jumps straight to the next symbol equal to the
// one at p, and each run is measured four bytes at a time; the visited runs
// are the same.  Ties keep the first run found (the farthest offset).
template <int S>
__device__ __forceinline__ void paper_match(const typename SymType<S>::T *sym, uint32_t k,
                                            const BufDesc &A, uint32_t p, uint32_t &best,
                                            uint32_t &bd) {
  const uint32_t end = min(k, p + A.M);
  const auto c = sym[p];
  best = 0;
  bd = 0;
  uint32_t w = p > A.W ? p - A.W : 0;
  while (true) {
    w = next_equal<S>(sym, w, p, c);
    if (w >= p) break;
    const uint32_t cap = min(p - w, end - p);
    const uint32_t l = extend_words<S>(reinterpret_cast<const uint8_t *>(sym), p, p - w, cap);
    if (l > best) {
      best = l;
      bd = p - w;
    }
    if (l == cap) break;  // the run reached p or the look-ahead end
    w += l + 1;
  }
}

// Exact longest match at p by the whole warp (fallback for positions whose
// chain exceeded the work cap): lanes hold the offsets d = lane + 1 + 32 j
// and advance the match one symbol per step, dropping offsets whose symbol
// differs or that reached d <= length (length <= offset), until none is
// left; the longest survives, the smallest offset breaks ties (warp min).
template <int S, int NJ>
__device__ __forceinline__ void window_match(const typename SymType<S>::T *sym,
                                             uint32_t k, const BufDesc &A,
                                             uint32_t p, uint32_t lane,
                                             uint32_t &L_out, uint32_t &d_out) {
  using Sym = typename SymType<S>::T;
  const uint32_t cap = min(A.M, k - p);
  const uint32_t dlim = min(A.W, p);
  uint32_t alive = 0;
#pragma unroll
  for (int j = 0; j < NJ; ++j)
    if (lane + 1 + 32 * j <= dlim) alive |= 1u << j;
  uint32_t L = 0;
  while (L < cap) {
    const Sym c = sym[p + L];
    uint32_t eq = 0;
#pragma unroll
    for (int j = 0; j < NJ; ++j) {
      const int idx = static_cast<int>(p + L) - static_cast<int>(lane + 1 + 32 * j);
      eq |= static_cast<uint32_t>(sym[idx < 0 ? 0 : idx] == c) << j;
    }
    // offsets d <= L drop out (length <= offset) unless matches may overlap
    const uint32_t jmin = (L > lane) ? ((L - lane - 1) >> 5) + 1 : 0;
    const uint32_t capm = A.match == kMatchOverlap ? kFull : (jmin >= 32 ? 0u : (kFull << jmin));
    const uint32_t nxt = alive & eq & capm;
    if (!__any_sync(kFull, nxt != 0)) break;
    alive = nxt;
    ++L;
  }
  const uint32_t mine = alive ? lane + 1 + 32 * (__ffs(alive) - 1) : kFull;
  L_out = L;
  d_out = L ? __reduce_min_sync(kFull, mine) : 0;
}

// Index of the (n+1)-th set bit of `bits` (n < popc(bits)): the smallest b
// with more than n set bits in bits[0..b].
__device__ __forceinline__ uint32_t nth_set_bit(uint32_t bits, uint32_t n) {
  uint32_t lo = 0;
#pragma unroll
  for (uint32_t step = 16; step > 0; step >>= 1) {
    const uint32_t t = lo + step - 1;  // candidate: is the answer above t?
    const uint32_t upto = t >= 31 ? kFull : ((2u << t) - 1u);
    if (static_cast<uint32_t>(__popc(bits & upto)) <= n) lo += step;
  }
  return lo;
}

// Number of lanes whose (ascending) value v is below x.
__device__ __forceinline__ uint32_t count_below(uint32_t v, uint32_t x) {
  uint32_t lo = 0;
#pragma unroll
  for (uint32_t step = 16; step > 0; step >>= 1) {
    const uint32_t y = __shfl_sync(kFull, v, lo + step - 1);
    if (y < x) lo += step;
  }
  const uint32_t top = __shfl_sync(kFull, v, 31);  // every lane takes part
  if (lo == 31 && top < x) lo = 32;
  return lo;
}

// First marked position >= p (k if none).
__device__ __forceinline__ uint32_t next_marked(const uint32_t *maybe, uint32_t p,
                                                uint32_t k) {
  if (p >= k) return k;
  const uint32_t nw = (k + 31) / 32;
  uint32_t w = p >> 5;
  uint32_t bits = maybe[w] & (kFull << (p & 31));
  while (!bits && ++w < nw) bits = maybe[w];
  return bits ? min(k, (w << 5) + __ffs(bits) - 1) : k;
}

__device__ __forceinline__ uint32_t warp_excl_scan(uint32_t x, uint32_t lane,
                                                   uint32_t &total) {
  uint32_t incl = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(kFull, incl, o);
    if (lane >= static_cast<uint32_t>(o)) incl += y;
  }
  total = __shfl_sync(kFull, incl, 31);
  return incl - x;
}

// Step 3: greedy parse of one chunk.  The walk decides the tokens and
// records only the pointers: bit q of `pbits` marks a pointer at position q,
// and the pointers' payload bytes (length, offset - 1) are listed in order
// in `list` (1 + offB bytes each; the payload staging area holds any chunk's
// list, since a pointer's bytes are part of the record's worst case).
// Literals are not copied here: the record is written in one pass once its
// place is known (emit_record, step 6).
//
// The marked positions are taken 32 at a time: lane i evaluates the i-th
// next marked position with chain_match (exact).  The parse through the
// batch is then a chain over lanes: from lane i (coding position q_i) it
// moves to the first marked position at or after q_i + len (pointer of
// len >= m) or q_i + 1 (literal); the unmarked positions in between are
// literals and marked positions jumped over are covered.  Pointer doubling
// over the lanes' successors finds the visited lanes; warp sums give the
// batch's token count and payload bytes (the local, first pass of the
// two-pass prefix sum of section 3.2.2, per batch).
template <int S, int NJ, bool WIDE>
__device__ __forceinline__ void greedy_walk(const typename SymType<S>::T *sym,
                                            uint32_t k, const BufDesc &A,
                                            const CompressSmem &sm, const uint32_t *maybe,
                                            const Links<WIDE> &links, uint32_t *pbits,
                                            uint8_t *list, uint32_t lane,
                                            uint32_t &ntok_out, uint32_t &pay_out,
                                            uint32_t &nptr_out, bool &sane) {
  const uint32_t list_cap = sm.pay_bytes;
  sane = true;
  const uint32_t nw = (k + 31) / 32;
  const uint32_t tsz_match = 1 + A.offB;
  for (uint32_t i = lane; i < nw; i += 32) pbits[i] = 0;
  __syncwarp();
  uint32_t p = 0, ntok = 0, pb = 0, np = 0;
  while (p < k) {
    const uint32_t q0 = next_marked(maybe, p, k);
    if (q0 > p) {  // run of literals
      ntok += q0 - p;
      pb += (q0 - p) * S;
      p = q0;
      if (p >= k) break;
    }
    // batch: lane i <- i-th marked position >= p (32 mark words at a time,
    // a warp scan of their popcounts locates each lane's target)
    uint32_t mypos = k, seen = 0;
    for (uint32_t w0 = p >> 5; w0 < nw && seen < 32; w0 += 32) {
      const uint32_t w = w0 + lane;
      uint32_t bits = w < nw ? maybe[w] : 0u;
      if (w == (p >> 5)) bits &= kFull << (p & 31);
      const uint32_t cnt = __popc(bits);
      uint32_t tot;
      const uint32_t excl = warp_excl_scan(cnt, lane, tot);
      const uint32_t want = lane - seen;  // this lane's target among these words
      const uint32_t j = count_below(excl + cnt, want + 1);  // word holding it
      const uint32_t jb = __shfl_sync(kFull, bits, j < 32 ? j : 0);
      const uint32_t je = __shfl_sync(kFull, excl, j < 32 ? j : 0);
      if (lane >= seen && want < tot) mypos = ((w0 + j) << 5) + nth_set_bit(jb, want - je);
      seen += tot;
    }
    const uint32_t nvalid = min(seen, 32u);
    const bool valid = lane < nvalid;
    uint32_t L = 0, bd = 0;
    bool resolved = true;
    if (valid) {
      if (A.match == kMatchPaper) paper_match<S>(sym, k, A, mypos, L, bd);
      else resolved = chain_match<S, WIDE>(sym, k, A, links, mypos, L, bd);
    }
    const uint32_t unres = __ballot_sync(kFull, !resolved);
    uint32_t nxt = valid ? mypos + (L >= A.m ? L : 1u) : k;
    uint32_t succ = count_below(mypos, nxt);
    if (!valid) succ = 32;
    // visited lanes: the chain lane 0, succ(0), succ(succ(0)), ... found by
    // pointer doubling (lane t computes the t-th element)
    uint32_t jr = succ;  // succ^(2^r) of this lane, 32 = past the batch
    uint32_t x = 0;      // for lane t: succ^(t's low bits so far)(0)
#pragma unroll
    for (uint32_t r = 0; r < 5; ++r) {
      const uint32_t xr = __shfl_sync(kFull, jr, x < 32 ? x : 0);
      if ((lane >> r) & 1u) x = x < 32 ? xr : 32;
      const uint32_t nj = __shfl_sync(kFull, jr, jr < 32 ? jr : 0);
      jr = jr < 32 ? nj : 32;
    }
    uint32_t visited = __reduce_or_sync(kFull, x < nvalid ? (1u << x) : 0u);
    // serial chase, only when a visited lane still needs the exact fallback
    uint32_t v = (visited & unres) ? 0 : nvalid;
    if (v == 0) visited = 0;
    while (v < nvalid) {
      visited |= 1u << v;
      if ((unres >> v) & 1u) {
        uint32_t tl, td;
        const uint32_t pos_v = __shfl_sync(kFull, mypos, v);
        window_match<S, NJ>(sym, k, A, pos_v, lane, tl, td);
        const uint32_t nv = pos_v + (tl >= A.m ? tl : 1u);
        const uint32_t sv = count_below(mypos, nv);
        if (lane == v) {
          L = tl;
          bd = td;
          nxt = nv;
          succ = sv;
        }
      }
      v = __shfl_sync(kFull, succ, v);
    }
    const uint32_t lastv = 31u - __clz(visited);
    const uint32_t nxt_last = __shfl_sync(kFull, nxt, lastv);
    const uint32_t after = next_marked(maybe, nxt_last, k);
    const bool isv = (visited >> lane) & 1u;
    const uint32_t succ_pos = __shfl_sync(kFull, mypos, succ < 32 ? succ : lane);
    const uint32_t run_end = (lane == lastv) ? after : succ_pos;
    const uint32_t run = isv ? run_end - nxt : 0u;  // literals after this lane's token
    const bool is_match = isv && L >= A.m;
    const uint32_t mmask = __ballot_sync(kFull, is_match);
    const uint32_t tot_t = __reduce_add_sync(kFull, isv ? 1u + run : 0u);
    const uint32_t tot_b =
        __reduce_add_sync(kFull, isv ? (is_match ? tsz_match : S) + run * S : 0u);
    const uint32_t nb = __popc(mmask);
    // consistency guard: the batch must stay inside the chunk and the list
    // (always true for a correct parse)
    if (ntok + tot_t > k || after > k || nxt_last > k || tsz_match * (np + nb) > list_cap) {
      sane = false;
      break;
    }
    if (is_match && GLZ_OK(mypos < k && tsz_match * (np + __popc(mmask & lanemask_lt(lane)) + 1) <= list_cap)) {
      uint8_t *o = list + tsz_match * (np + __popc(mmask & lanemask_lt(lane)));
      o[0] = static_cast<uint8_t>(L);
      o[1] = static_cast<uint8_t>((bd - 1) & 0xFF);
      if (A.offB == 2) o[2] = static_cast<uint8_t>((bd - 1) >> 8);
      atomicOr(&pbits[mypos >> 5], 1u << (mypos & 31));
    }
    ntok += tot_t;
    pb += tot_b;
    np += nb;
    p = after;
  }
  __syncwarp();
  ntok_out = ntok;
  pay_out = pb;
  nptr_out = np;
}

// Step 6 for a record with pointers: the flags (to fdst), then the payload
// and a stream-version-2 tail (to pdst), written in one pass over the
// chunk's positions, 32 at a time (lane = position).  The destinations are
// either the record's place (the stream, or a parking slot), or -- when a
// pointer's payload bytes never exceed the input bytes it covers (S * m >=
// 1 + offB) -- the shared memory it reads: the payload over the staged
// chunk (a token's payload never starts after its position's input, so
// nothing not yet read is overwritten) and the flags over the pointer
// bitmap (token t's flag word is written only once the bitmap word of
// position t has been read).  A position is a pointer start (its bit in
// pbits; its payload bytes are the next entry of `list`), inside the
// pointer that covers it (no token), or a literal (its S input bytes).  The
// owning pointer of a position is the last pointer start at or before it
// (a bit scan; one that began in an earlier round is carried).  Each
// token's payload offset and index follow from popcounts over the round
// (the local prefix sum of section 3.2.2); the flag bits of up to 32
// tokens per round are gathered with two warp ORs.  Returns false when the
// pass does not produce exactly (ntok, pay) (never for a correct walk).
template <int S>
__device__ __forceinline__ bool emit_record(uint8_t *fdst, uint8_t *payload, const uint8_t *inb,
                                            uint32_t k, uint32_t tail, const uint32_t *pbits,
                                            const uint8_t *list, uint32_t offB, uint32_t ntok,
                                            uint32_t pay, uint32_t fcap, uint32_t pcap,
                                            uint32_t lane) {
  const uint32_t tsz = 1 + offB;
  const uint32_t fb = (ntok + 7) / 8;
  const uint32_t lt = lanemask_lt(lane), le = lt | (1u << lane);
  uint32_t pbase = 0, tbase = 0, obase = 0;
  uint32_t cend = 0;   // end of the last pointer started before this round
  uint32_t fword = 0;  // flag bits of the current flag word (tokens 32*(tbase/32) ...)
  for (uint32_t r0 = 0; r0 < k; r0 += 32) {
    const uint32_t j = r0 + lane;
    const bool act = j < k;
    const uint32_t pw = pbits[r0 >> 5];
    const bool ps = (pw >> lane) & 1u;
    const uint32_t ord = obase + __popc(pw & lt);
    uint32_t tok = 0;  // this lane's pointer token bytes
    if (ps) {
      const uint8_t *e = list + tsz * ord;
      tok = e[0] | (static_cast<uint32_t>(e[1]) << 8) |
            (offB == 2 ? static_cast<uint32_t>(e[2]) << 16 : 0u);
    }
    const uint32_t mb = pw & le;
    const uint32_t ol = (31u - __clz(mb)) & 31u;
    const uint32_t oend = __shfl_sync(kFull, j + (tok & 0xFFu), ol);
    const uint32_t end_own = mb ? oend : cend;
    cend = __shfl_sync(kFull, end_own, 31);
    const bool lit = act && !ps && j >= end_own;
    const uint32_t litm = __ballot_sync(kFull, lit);
    const uint32_t tokm = litm | pw;
    const uint32_t po = pbase + S * __popc(litm & lt) + tsz * __popc(pw & lt);
    uint32_t v = 0;
    if (lit) {
      if constexpr (S == 1) v = inb[j];
      else if constexpr (S == 2) v = reinterpret_cast<const uint16_t *>(inb)[j];
      else v = reinterpret_cast<const uint32_t *>(inb)[j];
    }
    __syncwarp();  // every read of the round before any write (in place)
    if (lit && GLZ_OK(po + S <= pcap)) {
#pragma unroll
      for (uint32_t i = 0; i < S; ++i) payload[po + i] = static_cast<uint8_t>(v >> (8 * i));
    } else if (ps && GLZ_OK(po + tsz <= pcap)) {
      payload[po] = static_cast<uint8_t>(tok);
      payload[po + 1] = static_cast<uint8_t>(tok >> 8);
      if (offB == 2) payload[po + 2] = static_cast<uint8_t>(tok >> 16);
    }
    // flag bits of this round's tokens (at most 32: words w0 and w0 + 1)
    const uint32_t t = tbase + __popc(tokm & lt);
    const uint32_t w0 = tbase >> 5;
    const uint32_t lo = __reduce_or_sync(kFull, (ps && (t >> 5) == w0) ? 1u << (t & 31) : 0u);
    const uint32_t hi = __reduce_or_sync(kFull, (ps && (t >> 5) != w0) ? 1u << (t & 31) : 0u);
    fword |= lo;
    const uint32_t ntb = tbase + __popc(tokm);
    if ((ntb >> 5) != w0) {  // flag word w0 is complete
      if (lane < 4 && GLZ_OK(4 * w0 + lane < fcap))
        fdst[4 * w0 + lane] = static_cast<uint8_t>(fword >> (8 * lane));
      fword = hi;
    }
    pbase += S * __popc(litm) + tsz * __popc(pw);
    obase += __popc(pw);
    tbase = ntb;
    __syncwarp();
  }
  // the last, partial flag word (its bytes up to fb), the tail
  const uint32_t w0 = tbase >> 5;
  if (lane < 4 && 4 * w0 + lane < fb) fdst[4 * w0 + lane] = static_cast<uint8_t>(fword >> (8 * lane));
  const uint8_t tb = lane < tail ? inb[k * S + lane] : 0;
  __syncwarp();
  if (lane < tail && GLZ_OK(pbase + lane < pcap)) payload[pbase + lane] = tb;
  __syncwarp();
  return tbase == ntok && pbase + tail == pay;
}

// Step 5: decoupled look-back (single-pass scan over chunks).  Status word:
// bit 63 = inclusive prefix, bit 62 = aggregate only, low bits = value;
// 0 = not published yet.
constexpr unsigned long long kPrefix = 1ull << 63, kAgg = 1ull << 62;
constexpr unsigned long long kVal = kAgg - 1;
constexpr uint32_t kLookbackRounds = 8;  // windows of 32 per attempt
constexpr uint32_t kFreeSlot = 0xFFFFFFFFu;
constexpr uint32_t kLiteralRef = 1u << 31;  // parked record = zero flags + the input chunk

__device__ __forceinline__ void publish(unsigned long long *status, uint32_t c,
                                        unsigned long long flag, uint64_t v,
                                        uint32_t lane) {
  if (lane == 0) st_relaxed_u64(&status[c], flag | v);
}

// One non-blocking look-back attempt for chunk c: sum the published
// aggregates of the chunks before it back to the nearest published
// inclusive prefix.  False if a chunk it needs has not published yet (or
// the prefix is more than kLookbackRounds windows back).
__device__ __forceinline__ bool lookback_try(const unsigned long long *status,
                                             uint32_t c, uint32_t lane,
                                             uint64_t &excl,
                                             uint32_t max_rounds = kLookbackRounds) {
  excl = 0;
  if (c == 0) return true;
  int64_t base = static_cast<int64_t>(c) - 1;
  for (uint32_t r = 0; r < max_rounds; ++r) {
    const int64_t idx = base - static_cast<int64_t>(lane);
    const unsigned long long v = idx >= 0 ? ld_relaxed_u64(&status[idx]) : kPrefix;
    const uint32_t pref = __ballot_sync(kFull, (v & kPrefix) != 0);
    const uint32_t empty = __ballot_sync(kFull, v == 0);
    const uint32_t limit = pref ? __ffs(pref) - 1 : 31u;
    const uint32_t need = limit == 31 ? kFull : ((2u << limit) - 1u);
    if (empty & need) return false;
    excl += warp_sum_u64(lane <= limit ? (v & kVal) : 0ull);
    if (pref) return true;
    base -= 32;
  }
  return false;
}

// Blocking look-back: retry with exponential back-off; after `limit`
// attempts give up, raise kErrTimeout and return false.  Each attempt scans
// back as far as needed: every chunk publishes its aggregate as soon as its
// parse is done, so a full scan only ever waits on chunks still parsing, and
// chunk 0 always holds a prefix.
__device__ __forceinline__ bool lookback_wait(const unsigned long long *status,
                                              uint32_t c, uint32_t lane,
                                              uint32_t *err, uint64_t &excl,
                                              uint32_t limit) {
  uint32_t nap = 32;
  for (uint32_t spins = 0; spins < limit; ++spins) {
    if (lookback_try(status, c, lane, excl, 0xFFFFFFFFu)) return true;
    __nanosleep(nap);
    nap = min(nap * 2, 1024u);
  }
  if (lane == 0) atomicOr(err, kErrTimeout);
  return false;
}

// n zero bytes at dst (any alignment), by the warp.
__device__ __forceinline__ void warp_zero(uint8_t *dst, uint32_t n, uint32_t lane) {
  const uint32_t head =
      min(n, (4u - static_cast<uint32_t>(reinterpret_cast<uintptr_t>(dst) & 3u)) & 3u);
  if (lane < head) dst[lane] = 0;
  const uint32_t words = (n - head) >> 2;
  uint32_t *d32 = reinterpret_cast<uint32_t *>(dst + head);
  for (uint32_t j = lane; j < words; j += 32) d32[j] = 0;
  const uint32_t done = head + 4u * words;
  if (lane < n - done) dst[done + lane] = 0;
}

// Step 6 for a chunk whose global offset is known: publish its inclusive
// prefix, its index entry (every 64th chunk) and the stream size (last
// chunk).  Returns where its record goes, or nullptr when it must not be
// written (data not valid, or past the output capacity: kErrSmall).
__device__ __forceinline__ uint8_t *place_meta(const CompressArgs &A, const BufDesc &B,
                                               uint32_t c, uint64_t excl, uint64_t rec,
                                               bool data_ok, uint32_t lane) {
  publish(A.status + B.gbase, c, kPrefix, excl + rec, lane);
  if (c % kIndexStride == 0) {
    uint8_t *idx = B.out + kHeaderBytes + static_cast<uint64_t>(kTableEntry) * B.nc +
                   8ull * (c / kIndexStride);
    st_le_bytes(idx, excl, 8, lane);
  }
  const uint64_t dst = B.records_at + excl;
  if (c + 1 == B.nc && lane == 0) *B.out_bytes = dst + rec;
  if (!data_ok) return nullptr;
  if (dst + rec > B.cap) {
    if (lane == 0) atomicOr(A.err, kErrSmall);
    return nullptr;
  }
  return B.out + dst;
}

// Step 6 with the record's bytes in memory: (src1, n1) then (src2, n2);
// src1 == nullptr writes n1 zero bytes.
__device__ __forceinline__ void place_record(const CompressArgs &A, const BufDesc &B,
                                             uint32_t c, uint64_t excl, uint64_t rec,
                                             const uint8_t *src1, uint32_t n1,
                                             const uint8_t *src2, uint32_t n2,
                                             bool data_ok, uint32_t lane) {
  uint8_t *o = place_meta(A, B, c, excl, rec, data_ok, lane);
  if (!o) return;
  if (src1) warp_copy(o, src1, n1, lane);
  else warp_zero(o, n1, lane);
  if (n2) warp_copy(o + n1, src2, n2, lane);
}

__device__ __forceinline__ BufDesc buffer_of(const CompressArgs &A, uint32_t item) {
  return A.items ? A.items[item] : A.buf;
}

// A warp's shared-memory slice, TMA barrier phase and parking slots (lane s
// < park_slots describes slot s: chunk, buffer, record bytes).
struct WarpState {
  uint8_t *inb, *flags, *pay, *links_base, *slots;
  uint32_t *maybe;
  uint64_t *bar;
  uint32_t phase;
  uint32_t slot_c, slot_item, slot_rec;
  bool try_literal;  // the warp's previous chunk was all literals
};

// Parking slots of this warp whose chunk can now be placed are placed and
// freed; with `wait`, every occupied slot is placed (blocking).
__device__ __forceinline__ void drain_parked(const CompressArgs &A, WarpState &W,
                                             bool wait, uint32_t lane) {
  for (uint32_t sidx = 0; sidx < A.park_slots; ++sidx) {
    const uint32_t cs = __shfl_sync(kFull, W.slot_c, sidx);
    if (cs == kFreeSlot) continue;
    const uint32_t rs = __shfl_sync(kFull, W.slot_rec, sidx);
    const uint32_t is = __shfl_sync(kFull, W.slot_item, sidx);
    const BufDesc B = buffer_of(A, is);
    uint64_t excl;
    bool ok = lookback_try(A.status + B.gbase, cs, lane, excl);
    bool data_ok = true;
    if (!ok && wait) {
      ok = true;
      data_ok = lookback_wait(A.status + B.gbase, cs, lane, A.err, excl, A.spin_limit);
    }
    if (!ok) continue;
    if (rs & kLiteralRef) {
      // a record made of the chunk's own input bytes after zero flag bytes
      // (all literals), or of those bytes alone (a stored chunk)
      const uint32_t bytes = (cs + 1 < B.nc) ? B.C : static_cast<uint32_t>(B.n - uint64_t(cs) * B.C);
      const uint32_t rec = rs & ~kLiteralRef;
      place_record(A, B, cs, excl, rec, nullptr, rec - bytes,
                   B.in + static_cast<uint64_t>(cs) * B.C, bytes, data_ok, lane);
    } else {
      const uint8_t *slot = W.slots + static_cast<uint64_t>(sidx) * A.park_slot_bytes;
      place_record(A, B, cs, excl, rs, slot, rs, nullptr, 0, data_ok, lane);
    }
    if (lane == sidx) W.slot_c = kFreeSlot;
    __syncwarp();
  }
}

__device__ __forceinline__ void init_warp_state(const CompressArgs &A, uint8_t *smem,
                                                WarpState &W, uint32_t lane) {
  const uint32_t warp = threadIdx.x >> 5;
  uint8_t *ws = smem + warp * A.sm.per_warp;
  W.inb = ws + A.sm.in_off;
  W.flags = ws + A.sm.flags_off;
  W.pay = ws + A.sm.pay_off;
  W.links_base = ws + A.sm.prev_off;
  W.maybe = reinterpret_cast<uint32_t *>(ws + A.sm.maybe_off);
  W.bar = reinterpret_cast<uint64_t *>(ws + A.sm.mbar_off);
  if (lane == 0) {
    mbar_init(W.bar, 1);
    fence_mbar_init();
  }
  __syncwarp();
  W.phase = 0;
  const uint64_t gw = static_cast<uint64_t>(blockIdx.x) * (blockDim.x >> 5) + warp;
  W.slots = A.park + gw * A.park_slots * A.park_slot_bytes;
  W.slot_c = kFreeSlot;
  W.slot_item = 0;
  W.slot_rec = 0;
  W.try_literal = true;
}

__device__ __forceinline__ void write_header(const BufDesc &B, uint32_t lane) {
  uint32_t b = 0;
  switch (lane) {
    case 0: b = 'G'; break;
    case 1: b = 'L'; break;
    case 2: b = 'Z'; break;
    case 3: b = '1'; break;
    case 4: b = B.version == 2 ? 2u : 1u; break;
    case 5: b = B.S; break;
    case 6: b = B.offB; break;
    case 7: b = B.m; break;
    case 8: b = B.M; break;
    case 9: b = B.match == kMatchOverlap ? 1u : 0u; break;  // overlap flag (version 2)
    default:
      if (lane >= 12 && lane < 16) b = B.C >> (8 * (lane - 12));
      else if (lane >= 16 && lane < 20) b = B.W >> (8 * (lane - 16));
      else if (lane >= 20 && lane < 24) b = B.nc >> (8 * (lane - 20));
      else if (lane >= 24) b = static_cast<uint32_t>(B.n >> (8 * (lane - 24)));
  }
  B.out[lane] = static_cast<uint8_t>(b);
}

// Steps 1-6 for chunk c of buffer B (item `item` of a batch).  Returns false
// when the TMA copy never landed (the warp must stop: its barrier phase is
// unknown; the chunk was still published so no other warp waits on it).
template <int S, int NJ, bool WIDE>
__device__ __forceinline__ bool compress_chunk(const CompressArgs &A, const BufDesc &B,
                                               uint32_t item, uint32_t c, WarpState &W,
                                               uint32_t lane) {
  using Sym = typename SymType<S>::T;
  const Sym *sym = reinterpret_cast<const Sym *>(W.inb);
  const Links<WIDE> links{W.links_base};
  unsigned long long *status = A.status + B.gbase;
  if (c == 0) write_header(B, lane);

  // 1. stage the chunk
  const uint64_t chunk_at = static_cast<uint64_t>(c) * B.C;
  const uint32_t bytes = (c + 1 < B.nc) ? B.C : static_cast<uint32_t>(B.n - chunk_at);
  const uint32_t k = bytes / S;
  const uint8_t *src = B.in + chunk_at;
  const uint32_t bulk = B.in_aligned ? (bytes & ~15u) : 0u;
  if (lane == 0 && B.in_aligned) {
    // warm L2 for the chunk a wave of warps ahead (whichever warp takes it)
    const uint64_t ahead = static_cast<uint64_t>(c) + gridDim.x * (blockDim.x >> 5);
    if (ahead + 1 < B.nc) prefetch_l2(B.in + ahead * B.C, B.C);
  }
  if (bulk && lane == 0) {
    fence_proxy_async_smem();
    mbar_arrive_expect_tx(W.bar, bulk);
    bulk_g2s(W.inb, src, bulk, W.bar);
  }
  for (uint32_t i = bulk + lane; i < bytes; i += 32) W.inb[i] = src[i];
  bool staged = true;
  if (bulk) {
    staged = mbar_wait_bounded(W.bar, W.phase, A.spin_limit);
    W.phase ^= 1u;
    if (!staged && lane == 0) atomicOr(A.err, kErrTimeout);
  }
  __syncwarp();

  // 2. literal pre-check (its bitmap spans the links, flags and payload
  // areas, contiguous and unused until the chains; used for 2- and 4-byte
  // symbols when that gives at least 8 bits per position -- for 1-byte
  // symbols a key of three bytes repeats by chance often enough that the
  // check mostly gives up), else the candidate filter (hash table in the
  // payload area)
  const uint32_t bm_words = (A.sm.maybe_off - A.sm.prev_off) / 4;
  bool literal = false;
  // (tried when this warp's previous chunk was all literals: on data with
  // repeats the check would only give up, so it is not tried again until a
  // chunk without a match comes by)
  if (S >= 2 && W.try_literal && bm_words >= 16 && 4 * bm_words >= k)
    literal = literal_chunk<S>(sym, k, B, reinterpret_cast<uint32_t *>(W.links_base), bm_words,
                               W.maybe, lane);
  uint32_t marked = 0;
  if (!literal) {
    build_chains<S, WIDE>(sym, k, B, A.sm, reinterpret_cast<uint16_t *>(W.pay), W.maybe,
                          links, lane);
    for (uint32_t i = lane; i < (k + 31) / 32; i += 32) marked |= W.maybe[i];
  }
  __syncwarp();

  // 3. greedy parse: the walk records the pointers (a bitmap in the flags
  // area, their payload bytes listed in the payload area).  With no marked
  // position, or no pointer, the record is k literals: zero flags, then the
  // staged chunk itself.
  uint32_t ntok = k, pb = k * S, np = 0;
  bool sane = true;
  const uint8_t *payload = W.inb;
  uint32_t *pbits = reinterpret_cast<uint32_t *>(W.flags);
  if (__any_sync(kFull, marked != 0)) {
    greedy_walk<S, NJ, WIDE>(sym, k, B, A.sm, W.maybe, links, pbits, W.pay, lane, ntok, pb,
                             np, sane);
    if (!sane) {
      if (lane == 0) atomicOr(A.err, kErrInternal);
      ntok = k;
      pb = k * S;
      np = 0;
    }
  }
  // the record: 0 = zero flags + the staged chunk (all literals) or the
  // chunk alone (stored); 1 = pointers, emitted at the record's place;
  // 2 = pointers, emitted into shared memory (flags over the bitmap,
  // payload over the staged chunk)
  uint32_t kind = np != 0 ? 1u : 0u;
  W.try_literal = kind == 0;
  // 4. stream version 2, last chunk: the 1..S-1 bytes after the last whole
  // symbol follow the tokens as they are (in the staged chunk they already
  // follow the k symbols)
  const uint32_t tail = bytes - k * S;
  pb += tail;
  uint32_t fb = (ntok + 7) / 8;
  if (B.version == 2 && fb + pb >= bytes) {
    // stream version 2: a record that would not be smaller than the chunk is
    // replaced by the chunk's bytes, marked by a token count of 0
    ntok = 0;
    fb = 0;
    pb = bytes;
    payload = W.inb;
    kind = 0;
  }
  if (kind == 1 && S * B.m >= 1 + B.offB) {
    if (!emit_record<S>(W.flags, W.inb, W.inb, k, tail, pbits, W.pay, B.offB, ntok, pb,
                        A.sm.pay_off - A.sm.flags_off, A.sm.prev_off - A.sm.in_off, lane) &&
        lane == 0)
      atomicOr(A.err, kErrInternal);
    kind = 2;
  }
  const uint64_t rec = static_cast<uint64_t>(fb) + pb;
  const bool data_ok = staged && sane;
  // the record's bytes at o
  auto write_record = [&](uint8_t *o) {
    if (kind == 1) {
      if (!emit_record<S>(o, o + fb, W.inb, k, tail, pbits, W.pay, B.offB, ntok, pb, fb, pb,
                          lane) &&
          lane == 0)
        atomicOr(A.err, kErrInternal);
    } else {
      if (kind == 2) warp_copy(o, W.flags, fb, lane);
      else warp_zero(o, fb, lane);
      warp_copy(o + fb, payload, pb, lane);
    }
  };

  // 5. global offset: publish the aggregate at once, so that no other
  // chunk waits on this warp; write the record now if the offset is known,
  // else park it and move on (placed after a later chunk)
  if (c != 0) publish(status, c, kAgg, rec, lane);
  uint8_t *tab = B.out + kHeaderBytes + static_cast<uint64_t>(kTableEntry) * c;
  if (lane < 4)
    tab[lane] = static_cast<uint8_t>(ntok >> (8 * lane));
  else if (lane < 8)
    tab[lane] = static_cast<uint8_t>(pb >> (8 * (lane - 4)));
  drain_parked(A, W, false, lane);
  uint64_t excl;
  if (lookback_try(status, c, lane, excl)) {
    uint8_t *o = place_meta(A, B, c, excl, rec, data_ok, lane);
    if (o) write_record(o);
  } else {
    const uint32_t free_mask =
        __ballot_sync(kFull, lane < A.park_slots && W.slot_c == kFreeSlot);
    if (free_mask && data_ok) {
      const uint32_t sidx = __ffs(free_mask) - 1;
      // a record of zero flags and the chunk's input (all literals), or of
      // the input alone (stored), is parked by reference
      // (not the last chunk: a copy may read up to 3 bytes past its source)
      const bool by_ref = kind == 0 && c + 1 < B.nc;
      if (!by_ref && GLZ_OK(rec <= A.park_slot_bytes))
        write_record(W.slots + static_cast<uint64_t>(sidx) * A.park_slot_bytes);
      if (lane == sidx) {
        W.slot_c = c;
        W.slot_item = item;
        W.slot_rec = static_cast<uint32_t>(rec) | (by_ref ? kLiteralRef : 0u);
      }
    } else {
      const bool ok = lookback_wait(status, c, lane, A.err, excl, A.spin_limit);
      uint8_t *o = place_meta(A, B, c, excl, rec, data_ok && ok, lane);
      if (o) write_record(o);
    }
  }
  __syncwarp();
  return staged;
}

__device__ __forceinline__ uint32_t take_ticket(const CompressArgs &A, uint32_t lane) {
  uint32_t t = 0;
  if (lane == 0) t = atomicAdd(A.ticket, 1u) + A.first_ticket;
  return __shfl_sync(kFull, t, 0);
}

// Single buffer: the symbol size is a template parameter.
template <int S, int NJ>
__global__ void __launch_bounds__(256) compress_kernel(const CompressArgs A) {
  extern __shared__ __align__(128) uint8_t smem[];
  const uint32_t lane = threadIdx.x & 31;
  WarpState W;
  init_warp_state(A, smem, W, lane);
  while (true) {
    const uint32_t c = take_ticket(A, lane);
    if (c >= A.end_chunk) break;
    // one-byte links exactly when W <= 256, which is when NJ <= 8
    if (!compress_chunk<S, NJ, (NJ > 8)>(A, A.buf, 0, c, W, lane)) break;
  }
  drain_parked(A, W, true, lane);
  if (lane == 0) checked_fold(A.err);
}

// Buffer holding global chunk g: the last item whose first chunk is <= g,
// found by a 32-way search (one probe per lane per round).
__device__ __forceinline__ uint32_t find_item(const CompressArgs &A, uint64_t g,
                                              uint32_t lane) {
  uint32_t lo = 0, hi = A.n_items;  // answer in [lo, hi)
  while (hi - lo > 1) {
    const uint32_t step = (hi - lo + 31) / 32;
    const uint32_t idx = lo + lane * step;
    const bool le = idx < hi && A.item_base[idx] <= g;
    const uint32_t cnt = __popc(__ballot_sync(kFull, le));  // >= 1: lane 0 probes lo
    const uint32_t nlo = lo + (cnt - 1) * step;
    hi = min(hi, nlo + step);
    lo = nlo;
  }
  return lo;
}

// Batch: work items are the chunks of all buffers in order; each buffer
// carries its own parameters, so the symbol size is dispatched per chunk.
template <int NJ>
__global__ void __launch_bounds__(256) compress_batch_kernel(const CompressArgs A) {
  extern __shared__ __align__(128) uint8_t smem[];
  const uint32_t lane = threadIdx.x & 31;
  WarpState W;
  init_warp_state(A, smem, W, lane);
  while (true) {
    const uint32_t g = take_ticket(A, lane);
    if (g >= A.total_chunks) break;
    const uint32_t item = find_item(A, g, lane);
    const BufDesc B = A.items[item];
    const uint32_t c = static_cast<uint32_t>(g - B.gbase);
    bool ok;
    if constexpr (NJ > 8) {
      if (B.W > 256) {
        switch (B.S) {
          case 1: ok = compress_chunk<1, NJ, true>(A, B, item, c, W, lane); break;
          case 2: ok = compress_chunk<2, NJ, true>(A, B, item, c, W, lane); break;
          default: ok = compress_chunk<4, NJ, true>(A, B, item, c, W, lane); break;
        }
      } else {
        switch (B.S) {
          case 1: ok = compress_chunk<1, NJ, false>(A, B, item, c, W, lane); break;
          case 2: ok = compress_chunk<2, NJ, false>(A, B, item, c, W, lane); break;
          default: ok = compress_chunk<4, NJ, false>(A, B, item, c, W, lane); break;
        }
      }
    } else {
      switch (B.S) {
        case 1: ok = compress_chunk<1, NJ, false>(A, B, item, c, W, lane); break;
        case 2: ok = compress_chunk<2, NJ, false>(A, B, item, c, W, lane); break;
        default: ok = compress_chunk<4, NJ, false>(A, B, item, c, W, lane); break;
      }
    }
    if (!ok) break;
  }
  drain_parked(A, W, true, lane);
  if (lane == 0) checked_fold(A.err);
}

}  // namespace glz
