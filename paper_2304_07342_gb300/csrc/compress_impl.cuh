// compress_impl.cuh -- the fused compression kernel (one warp per chunk).
//
// gpuLZ splits compression into Kernel I (match + local prefix sum +
// encode, section 3.3.2), Kernel II (global prefix sum, 3.3.3) and Kernel
// III (deflate, 3.3.4).  Here all of it is one persistent kernel; each warp
// takes the next chunk from a work counter and
//   1. stages the chunk into its shared-memory slice (1-D TMA bulk copy);
//   2. marks the positions where a match of >= m symbols can exist, with a
//      last-occurrence hash table over the first min(m, 8/S) symbols
//      (__match_any_sync resolves collisions inside a 32-position slab);
//      the filter is conservative, so skipping unmarked positions as
//      literals leaves the greedy parse unchanged;
//   3. walks the greedy parse (section 2.2 steps 1-6): at a marked position
//      the lanes hold the candidate offsets d = lane+1+32j and advance the
//      match one symbol per step, dropping offsets whose symbol differs or
//      that reached d <= length (length <= offset, section 3.3.2), until no
//      candidate survives; the longest length wins, then the smallest
//      offset (warp min).  Tokens are appended to a staging record in
//      shared memory -- the running byte count is the local (first) pass of
//      the two-pass prefix sum (section 3.2.2);
//   4. obtains its record's global offset from a decoupled look-back over
//      the chunks before it (the second pass) -- bounded spins, no extra
//      kernel, no per-symbol data in HBM;
//   5. writes its table entry, index entry and record at the final offset.
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

// Step 2: one bit per position, set where a match of >= m symbols may
// start.  A position p can only have such a match if the same first
// g = min(m, 8/S) symbols occur at some q in [p-W, p-1]; the table keeps,
// per hash of those g symbols, the last position inserted, so "last
// occurrence older than W" proves there is none.
template <int S>
__device__ __forceinline__ void mark_candidates(const typename SymType<S>::T *sym,
                                                uint32_t k, const CompressArgs &A,
                                                uint16_t *table, uint32_t *maybe,
                                                uint32_t lane) {
  const uint32_t H = 1u << A.sm.hash_log2;
  // "last position" = p - (W + 1) for every p: never within the window
  const uint32_t init16 = static_cast<uint16_t>(0u - A.W - 1u);
  const uint32_t init32 = init16 | (init16 << 16);
  uint32_t *t32 = reinterpret_cast<uint32_t *>(table);
  for (uint32_t i = lane; i < H / 2; i += 32) t32[i] = init32;
  __syncwarp();

  const uint32_t g = min(A.m, 8u / S);
  const uint32_t shift = 64u - A.sm.hash_log2;
  const uint32_t lt = lanemask_lt(lane);
  const uint32_t nslab = (k + 31) / 32;
  for (uint32_t s = 0; s < nslab; ++s) {
    const uint32_t p = s * 32 + lane;
    const bool ok = p + A.m <= k;  // room for m symbols
    uint64_t key = 0;
    if (ok) {
#pragma unroll
      for (uint32_t i = 0; i < 8u / S; ++i)
        if (i < g) key |= static_cast<uint64_t>(sym[p + i]) << (8 * S * i);
    }
    const uint32_t h =
        static_cast<uint32_t>((key * 0x9E3779B97F4A7C15ull) >> shift);
    const uint32_t grp = __match_any_sync(kFull, ok ? h : (0x10000u + lane));
    const uint32_t lower = grp & lt;
    uint32_t dist;
    if (lower)
      dist = lane - (31u - __clz(lower));  // nearest earlier lane, same hash
    else
      dist = static_cast<uint16_t>(p - table[h]);
    __syncwarp();
    if (ok && (grp >> lane) == 1u) table[h] = static_cast<uint16_t>(p);
    const uint32_t bits = __ballot_sync(kFull, ok && dist <= A.W);
    if (lane == 0) maybe[s] = bits;
    __syncwarp();
  }
}

__device__ __forceinline__ void warp_copy_bytes(uint8_t *dst, const uint8_t *src,
                                                uint32_t nbytes, uint32_t lane) {
  for (uint32_t i = lane; i < nbytes; i += 32) dst[i] = src[i];
}

// Step 3: greedy parse of one chunk into (flags, payload) staging.
template <int S, int NJ>
__device__ __forceinline__ void greedy_walk(const typename SymType<S>::T *sym,
                                            uint32_t k, const CompressArgs &A,
                                            const uint32_t *maybe, uint8_t *flags,
                                            uint8_t *pay, uint32_t lane,
                                            uint32_t &ntok_out, uint32_t &pay_out) {
  using Sym = typename SymType<S>::T;
  const uint8_t *in_bytes = reinterpret_cast<const uint8_t *>(sym);
  const uint32_t nw = (k + 31) / 32;
  uint32_t p = 0, ntok = 0, pb = 0;
  while (p < k) {
    // next marked position at or after p
    uint32_t w = p >> 5;
    uint32_t bits = maybe[w] & (kFull << (p & 31));
    while (!bits && ++w < nw) bits = maybe[w];
    const uint32_t q = bits ? min(k, (w << 5) + __ffs(bits) - 1) : k;
    if (q > p) {  // run of literals
      const uint32_t nb = (q - p) * S;
      warp_copy_bytes(pay + pb, in_bytes + p * S, nb, lane);
      pb += nb;
      ntok += q - p;
      p = q;
      __syncwarp();
      continue;
    }
    // longest match at p over offsets d = lane + 1 + 32 j <= min(W, p)
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
      // offsets d <= L would read the look-ahead itself: drop them
      const uint32_t jmin = (L > lane) ? ((L - lane - 1) >> 5) + 1 : 0;
      const uint32_t capm = jmin >= 32 ? 0u : (kFull << jmin);
      const uint32_t nxt = alive & eq & capm;
      if (!__any_sync(kFull, nxt != 0)) break;
      alive = nxt;
      ++L;
    }
    if (L >= A.m) {
      const uint32_t mine = alive ? lane + 1 + 32 * (__ffs(alive) - 1) : kFull;
      const uint32_t d = __reduce_min_sync(kFull, mine);
      if (lane == 0) {
        flags[ntok >> 3] |= static_cast<uint8_t>(1u << (ntok & 7));
        pay[pb] = static_cast<uint8_t>(L);
        pay[pb + 1] = static_cast<uint8_t>((d - 1) & 0xFF);
        if (A.offB == 2) pay[pb + 2] = static_cast<uint8_t>((d - 1) >> 8);
      }
      pb += 1 + A.offB;
      p += L;
    } else {
      if (lane < S) pay[pb + lane] = in_bytes[p * S + lane];
      pb += S;
      p += 1;
    }
    ++ntok;
    __syncwarp();
  }
  ntok_out = ntok;
  pay_out = pb;
}

// Step 4: decoupled look-back (single-pass scan over chunks).  Status word:
// bit 63 = inclusive prefix, bit 62 = aggregate only, low bits = value;
// 0 = not published yet.  Returns the exclusive prefix of record bytes.
__device__ __forceinline__ uint64_t chunk_lookback(unsigned long long *status,
                                                   uint32_t c, uint64_t agg,
                                                   uint32_t lane, uint32_t *err,
                                                   bool &ok) {
  constexpr unsigned long long kPrefix = 1ull << 63, kAgg = 1ull << 62;
  constexpr unsigned long long kVal = kAgg - 1;
  ok = true;
  if (c == 0) {
    if (lane == 0) st_relaxed_u64(&status[0], kPrefix | agg);
    return 0;
  }
  if (lane == 0) st_relaxed_u64(&status[c], kAgg | agg);
  uint64_t excl = 0;
  int64_t base = static_cast<int64_t>(c) - 1;
  uint32_t spins = 0;
  while (true) {
    const int64_t idx = base - static_cast<int64_t>(lane);
    const unsigned long long v = idx >= 0 ? ld_relaxed_u64(&status[idx]) : kPrefix;
    const uint32_t pref = __ballot_sync(kFull, (v & kPrefix) != 0);
    const uint32_t empty = __ballot_sync(kFull, v == 0);
    const uint32_t limit = pref ? __ffs(pref) - 1 : 31u;
    const uint32_t need = limit == 31 ? kFull : ((2u << limit) - 1u);
    if (empty & need) {
      if (++spins > kSpinLimit) {
        ok = false;
        if (lane == 0) atomicOr(err, kErrTimeout);
        break;
      }
      __nanosleep(20);
      continue;
    }
    excl += warp_sum_u64(lane <= limit ? (v & kVal) : 0ull);
    if (pref) break;
    base -= 32;
  }
  // a timed-out chunk still publishes so that its successors do not wait
  if (lane == 0) st_relaxed_u64(&status[c], kPrefix | (excl + agg));
  return excl;
}

template <int S, int NJ>
__global__ void __launch_bounds__(256) compress_kernel(const CompressArgs A) {
  using Sym = typename SymType<S>::T;
  extern __shared__ __align__(128) uint8_t smem[];
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t warp = threadIdx.x >> 5;
  uint8_t *ws = smem + warp * A.sm.per_warp;
  uint8_t *inb = ws + A.sm.in_off;
  uint8_t *flags = ws + A.sm.flags_off;
  uint8_t *pay = ws + A.sm.pay_off;
  uint32_t *maybe = reinterpret_cast<uint32_t *>(ws + A.sm.maybe_off);
  uint64_t *bar = reinterpret_cast<uint64_t *>(ws + A.sm.mbar_off);
  const Sym *sym = reinterpret_cast<const Sym *>(inb);

  if (lane == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
  }
  __syncwarp();
  uint32_t phase = 0;

  while (true) {
    uint32_t c = 0;
    if (lane == 0) c = atomicAdd(A.ticket, 1u);
    c = __shfl_sync(kFull, c, 0);
    if (c >= A.nc) break;

    if (c == 0) {  // header
      uint32_t b = 0;
      switch (lane) {
        case 0: b = 'G'; break;
        case 1: b = 'L'; break;
        case 2: b = 'Z'; break;
        case 3: b = '1'; break;
        case 4: b = 1; break;
        case 5: b = A.S; break;
        case 6: b = A.offB; break;
        case 7: b = A.m; break;
        case 8: b = A.M; break;
        default:
          if (lane >= 12 && lane < 16) b = A.C >> (8 * (lane - 12));
          else if (lane >= 16 && lane < 20) b = A.W >> (8 * (lane - 16));
          else if (lane >= 20 && lane < 24) b = A.nc >> (8 * (lane - 20));
          else if (lane >= 24) b = static_cast<uint32_t>(A.n >> (8 * (lane - 24)));
      }
      A.out[lane] = static_cast<uint8_t>(b);
    }

    // 1. stage the chunk
    const uint64_t chunk_at = static_cast<uint64_t>(c) * A.C;
    const uint32_t bytes =
        (c + 1 < A.nc) ? A.C : static_cast<uint32_t>(A.n - chunk_at);
    const uint32_t k = bytes / S;
    const uint8_t *src = A.in + chunk_at;
    const uint32_t bulk = A.in_aligned ? (bytes & ~15u) : 0u;
    if (bulk && lane == 0) {
      fence_proxy_async_smem();
      mbar_arrive_expect_tx(bar, bulk);
      bulk_g2s(inb, src, bulk, bar);
    }
    for (uint32_t i = bulk + lane; i < bytes; i += 32) inb[i] = src[i];
    bool staged = true;
    if (bulk) {
      staged = mbar_wait_bounded(bar, phase);
      phase ^= 1u;
      if (!staged && lane == 0) atomicOr(A.err, kErrTimeout);
    }
    __syncwarp();

    // 2. candidate filter (hash table lives in the payload staging area)
    mark_candidates<S>(sym, k, A, reinterpret_cast<uint16_t *>(pay), maybe, lane);
    const uint32_t fbytes_max = (k + 7) / 8;
    for (uint32_t i = lane; i < fbytes_max; i += 32) flags[i] = 0;
    __syncwarp();

    // 3. greedy parse + local offsets
    uint32_t ntok, pb;
    greedy_walk<S, NJ>(sym, k, A, maybe, flags, pay, lane, ntok, pb);
    const uint32_t fb = (ntok + 7) / 8;
    const uint64_t rec = static_cast<uint64_t>(fb) + pb;

    // 4. global offset
    bool ok;
    const uint64_t excl = chunk_lookback(A.status, c, rec, lane, A.err, ok);

    // 5. table, index, record
    uint8_t *tab = A.out + kHeaderBytes + static_cast<uint64_t>(kTableEntry) * c;
    if (lane < 4)
      tab[lane] = static_cast<uint8_t>(ntok >> (8 * lane));
    else if (lane < 8)
      tab[lane] = static_cast<uint8_t>(pb >> (8 * (lane - 4)));
    if (c % kIndexStride == 0) {
      uint8_t *idx = A.out + kHeaderBytes + static_cast<uint64_t>(kTableEntry) * A.nc +
                     8ull * (c / kIndexStride);
      st_le_bytes(idx, excl, 8, lane);
    }
    const uint64_t dst = A.records_at + excl;
    if (ok && staged) {
      if (dst + rec > A.cap) {
        if (lane == 0) atomicOr(A.err, kErrSmall);
      } else {
        uint8_t *o = A.out + dst;
        for (uint32_t i = lane; i < fb; i += 32) o[i] = flags[i];
        for (uint32_t i = lane; i < pb; i += 32) o[fb + i] = pay[i];
      }
    }
    if (c + 1 == A.nc && lane == 0) *A.out_bytes = dst + rec;
    __syncwarp();
    // a copy that never landed leaves the barrier phase unknown: stop here
    // (the chunk was still published, so no other warp waits on it)
    if (!staged) break;
  }
}

}  // namespace glz
