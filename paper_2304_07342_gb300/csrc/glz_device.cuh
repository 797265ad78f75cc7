// glz_device.cuh -- small device helpers: inline PTX for the mbarrier/TMA
// bulk-copy path, relaxed global atomics for the look-back status words,
// and warp utilities.  Product code only.
#pragma once

#include <cstdint>

#include "glz_common.h"

namespace glz {

constexpr uint32_t kFull = 0xFFFFFFFFu;

// Bounds-checked build (compiled with -DLZ_CHECKED): GLZ_OK(cond) guards a
// shared- or global-memory access whose index the kernels compute; a false
// condition records a violation in this translation unit's device word and
// the access is skipped (no trap).  Each kernel folds the word into the
// context's error word (kErrInternal, LZ_ERR_INTERNAL from lz_sync) when
// it finishes.  In the normal build GLZ_OK is `true` and costs nothing.
#ifdef LZ_CHECKED
static __device__ unsigned int g_checked_violations;
__device__ __forceinline__ bool checked_ok(bool ok) {
  if (!ok) atomicAdd(&g_checked_violations, 1u);
  return ok;
}
#define GLZ_OK(cond) ::glz::checked_ok(cond)
__device__ __forceinline__ void checked_fold(uint32_t *err) {
  if (*reinterpret_cast<volatile unsigned int *>(&g_checked_violations) != 0) atomicOr(err, kErrInternal);
}
#else
#define GLZ_OK(cond) true
__device__ __forceinline__ void checked_fold(uint32_t *) {}
#endif

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// ---- mbarrier + cp.async.bulk (1-D TMA) --------------------------------------

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(count)
               : "memory");
}

// Make the mbarrier initialisation visible to the async (TMA) proxy.
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Order this thread's earlier generic-proxy shared accesses before later
// async-proxy (TMA) accesses of the same bytes.
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar,
                                                      uint32_t bytes) {
  asm volatile(
      "mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(
          smem_addr(bar)),
      "r"(bytes)
      : "memory");
}

// Global -> shared bulk copy; bytes and both addresses multiples of 16.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src,
                                         uint32_t bytes, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes "
      "[%0], [%1], %2, [%3];" ::"r"(smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(done)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return done != 0;
}

// Bounded wait for phase `parity` of `bar`; false if `limit` polls ran out.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity,
                                                  uint32_t limit = kSpinLimit) {
  for (uint32_t i = 0; i < limit; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

// L2 prefetch of a global range (address and size multiples of 16).
__device__ __forceinline__ void prefetch_l2(const void *src, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes)
               : "memory");
}

// ---- relaxed device-scope status words -----------------------------------------

__device__ __forceinline__ void st_relaxed_u64(unsigned long long *p,
                                               unsigned long long v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v)
               : "memory");
}

__device__ __forceinline__ unsigned long long ld_relaxed_u64(
    const unsigned long long *p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];"
               : "=l"(v)
               : "l"(p)
               : "memory");
  return v;
}

// ---- warp utilities ----------------------------------------------------------

__device__ __forceinline__ uint32_t lanemask_lt(uint32_t lane) {
  return (1u << lane) - 1u;
}

__device__ __forceinline__ unsigned long long warp_sum_u64(
    unsigned long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}

// Warp copy of n bytes between any two addresses (shared or global).  When
// source and destination share their alignment modulo 16 (and n >= 256) the
// body moves as 16-byte words.  Otherwise the
// destination is written in aligned 32-bit words, each assembled from two
// aligned source words with a funnel shift; unaligned head and tail bytes
// are copied singly.  Eight words per lane are loaded before any is stored,
// so a copy from global memory waits on one round trip per 1 KiB rather
// than per 128 bytes.  May read up to 3 bytes past the source range (the
// callers' source regions have that slack).  Source and destination must
// not overlap.
__device__ __forceinline__ void warp_copy(uint8_t *dst, const uint8_t *src,
                                          uint32_t n, uint32_t lane) {
  constexpr uint32_t U = 8;
  if ((((reinterpret_cast<uintptr_t>(dst) ^ reinterpret_cast<uintptr_t>(src)) & 15u) == 0) &&
      n >= 256) {
    // co-aligned: 16-byte words, four per lane in flight
    const uint32_t h16 =
        (16u - static_cast<uint32_t>(reinterpret_cast<uintptr_t>(dst) & 15u)) & 15u;
    if (lane < h16) dst[lane] = src[lane];
    const uint32_t q = (n - h16) >> 4;
    const uint4 *s16 = reinterpret_cast<const uint4 *>(src + h16);
    uint4 *d16 = reinterpret_cast<uint4 *>(dst + h16);
    uint32_t j = lane;
    for (; j + 96 < q; j += 128) {
      const uint4 a = s16[j], b = s16[j + 32], c = s16[j + 64], d = s16[j + 96];
      d16[j] = a;
      d16[j + 32] = b;
      d16[j + 64] = c;
      d16[j + 96] = d;
    }
    for (; j < q; j += 32) d16[j] = s16[j];
    const uint32_t done16 = h16 + 16u * q;
    if (lane < n - done16) dst[done16 + lane] = src[done16 + lane];
    return;
  }
  const uint32_t head =
      min(n, (4u - static_cast<uint32_t>(reinterpret_cast<uintptr_t>(dst) & 3u)) & 3u);
  if (lane < head) dst[lane] = src[lane];
  const uint32_t words = (n - head) >> 2;
  if (words) {
    const uint8_t *sb = src + head;
    const uint32_t sm = static_cast<uint32_t>(reinterpret_cast<uintptr_t>(sb) & 3u);
    const uint32_t *s32 = reinterpret_cast<const uint32_t *>(sb - sm);
    uint32_t *d32 = reinterpret_cast<uint32_t *>(dst + head);
    uint32_t j = lane;
    if (sm == 0) {
      for (; j + 32 * (U - 1) < words; j += 32 * U) {
        uint32_t v[U];
#pragma unroll
        for (uint32_t i = 0; i < U; ++i) v[i] = s32[j + 32 * i];
#pragma unroll
        for (uint32_t i = 0; i < U; ++i) d32[j + 32 * i] = v[i];
      }
      for (; j < words; j += 32) d32[j] = s32[j];
    } else {
      const uint32_t sh = 8u * sm;
      for (; j + 32 * (U - 1) < words; j += 32 * U) {
        uint32_t lo[U], hi[U];
#pragma unroll
        for (uint32_t i = 0; i < U; ++i) {
          lo[i] = s32[j + 32 * i];
          hi[i] = s32[j + 32 * i + 1];
        }
#pragma unroll
        for (uint32_t i = 0; i < U; ++i) d32[j + 32 * i] = __funnelshift_r(lo[i], hi[i], sh);
      }
      for (; j < words; j += 32) d32[j] = __funnelshift_r(s32[j], s32[j + 1], sh);
    }
  }
  const uint32_t done = head + 4u * words;
  if (lane < n - done) dst[done + lane] = src[done + lane];
}

// Little-endian byte stores/loads usable at any alignment.
__device__ __forceinline__ void st_le_bytes(uint8_t *dst, uint64_t v,
                                            uint32_t nbytes, uint32_t lane) {
  if (lane < nbytes) dst[lane] = static_cast<uint8_t>(v >> (8 * lane));
}

__device__ __forceinline__ uint64_t ld_le(const uint8_t *src,
                                          uint32_t nbytes) {
  uint64_t v = 0;
  for (uint32_t i = 0; i < nbytes; ++i) v |= static_cast<uint64_t>(src[i]) << (8 * i);
  return v;
}

}  // namespace glz
