/*
 * huffref.c -- CPU oracle for the Huffman stage after LZSS (the paper's
 * cuSZ use case, section 4.5).  TEST INFRASTRUCTURE ONLY (see huffref.h).
 *
 * Written for a reader to check by eye: a histogram, package-merge for the
 * length-limited code, canonical code assignment, then bit-by-bit writing
 * and reading.  No tables, no word tricks.
 */
#include "huffref.h"

#include <stdlib.h>
#include <string.h>

enum { H_OK = 0, H_EINVAL = 1, H_ESMALL = 2, H_ECORRUPT = 3 };

#define H_HEADER 16u
#define H_LENGTHS 256u
#define H_SUBS (HUFFREF_BLOCK / HUFFREF_SUB) /* 32 sub-blocks per block */

/* One item of a package-merge list: a leaf (a symbol) or a package of two
 * items of the next deeper list. */
typedef struct {
  uint64_t weight;
  int leaf;          /* 1: symbol `sym`; 0: package of child[0], child[1] */
  uint32_t sym;
  uint32_t child[2]; /* indices into the deeper list */
} h_item;

/* Package-merge (Larmore and Hirschberg, 1990) for an optimal prefix code
 * whose lengths do not exceed max_len.  The leaves are the present symbols
 * sorted by (count, value).  The deepest list holds the leaves; each
 * shallower list merges the leaves with the packages formed from
 * consecutive pairs of the list below (an odd last item is dropped),
 * ordered by weight, a leaf before a package of equal weight, packages in
 * the order they were formed.  The first 2n - 2 items of the shallowest
 * list are selected; a selected package selects both its children, and a
 * symbol's length is the number of lists in which it is selected. */
void huffref_lengths(const uint64_t *hist, uint32_t max_len, uint8_t *len) {
  memset(len, 0, 256);
  uint32_t n = 0, present[256];
  for (uint32_t s = 0; s < 256; ++s)
    if (hist[s]) present[n++] = s;
  if (n == 0) return;
  if (n == 1) {
    len[present[0]] = 1;
    return;
  }
  /* leaves sorted by (count, value): insertion sort, n <= 256 */
  for (uint32_t i = 1; i < n; ++i) {
    uint32_t s = present[i], j = i;
    while (j > 0 && (hist[present[j - 1]] > hist[s] ||
                     (hist[present[j - 1]] == hist[s] && present[j - 1] > s))) {
      present[j] = present[j - 1];
      --j;
    }
    present[j] = s;
  }
  h_item *lists[16];
  uint32_t count[16];
  for (uint32_t d = 0; d < max_len; ++d) lists[d] = (h_item *)malloc(sizeof(h_item) * 2 * n);
  /* lists[max_len - 1] is the deepest, lists[0] the shallowest */
  uint32_t deep = max_len - 1;
  for (uint32_t i = 0; i < n; ++i) {
    h_item it = {hist[present[i]], 1, present[i], {0, 0}};
    lists[deep][i] = it;
  }
  count[deep] = n;
  for (int d = (int)deep - 1; d >= 0; --d) {
    const h_item *below = lists[d + 1];
    uint32_t npk = count[d + 1] / 2, li = 0, pi = 0, out = 0;
    while (li < n || pi < npk) {
      uint64_t pw = pi < npk ? below[2 * pi].weight + below[2 * pi + 1].weight : 0;
      if (li < n && (pi >= npk || hist[present[li]] <= pw)) {
        h_item it = {hist[present[li]], 1, present[li], {0, 0}};
        lists[d][out++] = it;
        ++li;
      } else {
        h_item it = {pw, 0, 0, {2 * pi, 2 * pi + 1}};
        lists[d][out++] = it;
        ++pi;
      }
    }
    count[d] = out;
  }
  /* selection: the first 2n - 2 items of the shallowest list */
  uint8_t *sel[16];
  for (uint32_t d = 0; d < max_len; ++d) sel[d] = (uint8_t *)calloc(2 * n, 1);
  for (uint32_t i = 0; i < 2 * n - 2 && i < count[0]; ++i) sel[0][i] = 1;
  for (uint32_t d = 0; d < max_len; ++d) {
    for (uint32_t i = 0; i < count[d]; ++i) {
      if (!sel[d][i]) continue;
      const h_item *it = &lists[d][i];
      if (it->leaf) {
        len[it->sym] += 1;
      } else {
        sel[d + 1][it->child[0]] = 1;
        sel[d + 1][it->child[1]] = 1;
      }
    }
  }
  for (uint32_t d = 0; d < max_len; ++d) {
    free(lists[d]);
    free(sel[d]);
  }
}

/* Canonical codes: symbols in order of (length, value) take consecutive
 * code values; when the length grows by g the next value is shifted left
 * by g. */
void huffref_codes(const uint8_t *len, uint32_t *code) {
  memset(code, 0, 256 * sizeof(uint32_t));
  uint32_t next = 0, cur_len = 0;
  int first = 1;
  for (uint32_t l = 1; l <= 32; ++l) {
    for (uint32_t s = 0; s < 256; ++s) {
      if (len[s] != l) continue;
      if (first) {
        next = 0;
        first = 0;
      } else {
        next = (next + 1) << (l - cur_len);
      }
      cur_len = l;
      code[s] = next;
    }
  }
}

static void h_put_u32(uint8_t *p, uint32_t v) {
  for (int i = 0; i < 4; ++i) p[i] = (uint8_t)(v >> (8 * i));
}
static void h_put_u64(uint8_t *p, uint64_t v) {
  for (int i = 0; i < 8; ++i) p[i] = (uint8_t)(v >> (8 * i));
}
static uint32_t h_get_u32(const uint8_t *p) {
  uint32_t v = 0;
  for (int i = 0; i < 4; ++i) v |= (uint32_t)p[i] << (8 * i);
  return v;
}
static uint64_t h_get_u64(const uint8_t *p) {
  uint64_t v = 0;
  for (int i = 0; i < 8; ++i) v |= (uint64_t)p[i] << (8 * i);
  return v;
}

static uint64_t h_div_up(uint64_t a, uint64_t b) { return (a + b - 1) / b; }

uint64_t huffref_bound(uint64_t n) {
  uint64_t nb = h_div_up(n, HUFFREF_BLOCK);
  /* every byte at most HUFFREF_MAX_LEN bits, each block padded to words */
  return H_HEADER + H_LENGTHS + nb * 8u + nb * H_SUBS * 4u +
         h_div_up(n * HUFFREF_MAX_LEN, 32) * 4u + nb * 4u;
}

/* bit i of a block's bit string: bit 31 - (i % 32) of u32 word i / 32 */
static void h_put_bit(uint8_t *blk, uint64_t i, uint32_t b) {
  if (!b) return;
  uint64_t w = i / 32;
  uint32_t bit = 31u - (uint32_t)(i % 32);
  blk[4 * w + bit / 8] |= (uint8_t)(1u << (bit % 8));
}
static uint32_t h_get_bit(const uint8_t *blk, uint64_t i) {
  uint64_t w = i / 32;
  uint32_t bit = 31u - (uint32_t)(i % 32);
  return (blk[4 * w + bit / 8] >> (bit % 8)) & 1u;
}

int huffref_compress(const uint8_t *in, uint64_t n, uint8_t *out,
                     uint64_t cap, uint64_t *out_bytes) {
  uint64_t nb = h_div_up(n, HUFFREF_BLOCK);
  if (nb > 0xFFFFFFFFull) return H_EINVAL;
  uint64_t table_at = H_HEADER + H_LENGTHS;
  uint64_t subs_at = table_at + 8u * nb;
  uint64_t bits_at = subs_at + 4u * H_SUBS * nb;
  if (cap < bits_at) return H_ESMALL;
  memset(out, 0, (size_t)bits_at);
  memcpy(out, "GHF1", 4);
  h_put_u32(out + 4, HUFFREF_BLOCK);
  h_put_u64(out + 8, n);

  uint64_t hist[256] = {0};
  for (uint64_t i = 0; i < n; ++i) hist[in[i]]++;
  uint8_t len[256];
  uint32_t code[256];
  huffref_lengths(hist, HUFFREF_MAX_LEN, len);
  huffref_codes(len, code);
  memcpy(out + H_HEADER, len, 256);

  uint64_t pos = bits_at;
  for (uint64_t b = 0; b < nb; ++b) {
    uint64_t lo = b * HUFFREF_BLOCK;
    uint64_t hi = lo + HUFFREF_BLOCK < n ? lo + HUFFREF_BLOCK : n;
    uint64_t nbits = 0;
    for (uint64_t i = lo; i < hi; ++i) nbits += len[in[i]];
    uint64_t bytes = h_div_up(nbits, 32) * 4u;
    if (pos + bytes > cap) return H_ESMALL;
    uint8_t *blk = out + pos;
    memset(blk, 0, (size_t)bytes);
    uint64_t bit = 0;
    for (uint32_t s = 0; s < H_SUBS; ++s) {
      h_put_u32(out + subs_at + 4u * (H_SUBS * b + s), (uint32_t)bit);
      uint64_t slo = lo + (uint64_t)s * HUFFREF_SUB;
      uint64_t shi = slo + HUFFREF_SUB < hi ? slo + HUFFREF_SUB : hi;
      for (uint64_t i = slo; i < shi; ++i) {
        uint32_t l = len[in[i]], c = code[in[i]];
        for (uint32_t j = 0; j < l; ++j) h_put_bit(blk, bit++, (c >> (l - 1 - j)) & 1u);
      }
    }
    pos += bytes;
    h_put_u64(out + table_at + 8u * b, pos - bits_at);
  }
  *out_bytes = pos;
  return H_OK;
}

static int h_read_header(const uint8_t *in, uint64_t in_bytes, uint64_t *n) {
  if (in_bytes < H_HEADER + H_LENGTHS) return H_ECORRUPT;
  if (memcmp(in, "GHF1", 4) != 0 || h_get_u32(in + 4) != HUFFREF_BLOCK) return H_ECORRUPT;
  *n = h_get_u64(in + 8);
  return H_OK;
}

int huffref_decompressed_size(const uint8_t *in, uint64_t in_bytes,
                              uint64_t *n) {
  return h_read_header(in, in_bytes, n);
}

/* Decode by walking the canonical code one bit at a time: after reading l
 * bits the value v is a code of length l iff some symbol of length l has
 * code v. */
int huffref_decompress(const uint8_t *in, uint64_t in_bytes, uint8_t *out,
                       uint64_t cap, uint64_t *out_bytes) {
  uint64_t n;
  int rc = h_read_header(in, in_bytes, &n);
  if (rc != H_OK) return rc;
  if (cap < n) return H_ESMALL;
  const uint8_t *len = in + H_HEADER;
  uint64_t kraft = 0; /* sum of 2^(16 - len): a complete code gives 2^16 */
  uint32_t present = 0;
  for (uint32_t s = 0; s < 256; ++s) {
    if (len[s] > HUFFREF_MAX_LEN) return H_ECORRUPT;
    if (len[s]) {
      kraft += 1ull << (16 - len[s]);
      ++present;
    }
  }
  if (n > 0 && (present == 0 || (present == 1 ? kraft != (1ull << 15) : kraft != (1ull << 16))))
    return H_ECORRUPT;
  uint32_t code[256];
  huffref_codes(len, code);
  uint64_t nb = h_div_up(n, HUFFREF_BLOCK);
  uint64_t table_at = H_HEADER + H_LENGTHS;
  uint64_t subs_at = table_at + 8u * nb;
  uint64_t bits_at = subs_at + 4u * H_SUBS * nb;
  if (in_bytes < bits_at) return H_ECORRUPT;
  uint64_t pos = bits_at;
  for (uint64_t b = 0; b < nb; ++b) {
    uint64_t end = h_get_u64(in + table_at + 8u * b);
    if (end < pos - bits_at) return H_ECORRUPT;
    uint64_t bytes = end - (pos - bits_at);
    if (bytes % 4 || pos + bytes > in_bytes) return H_ECORRUPT;
    const uint8_t *blk = in + pos;
    uint64_t lo = b * HUFFREF_BLOCK;
    uint64_t hi = lo + HUFFREF_BLOCK < n ? lo + HUFFREF_BLOCK : n;
    uint64_t bit = 0;
    for (uint32_t s = 0; s < H_SUBS; ++s) {
      if (h_get_u32(in + subs_at + 4u * (H_SUBS * b + s)) != bit) return H_ECORRUPT;
      uint64_t slo = lo + (uint64_t)s * HUFFREF_SUB;
      uint64_t shi = slo + HUFFREF_SUB < hi ? slo + HUFFREF_SUB : hi;
      for (uint64_t i = slo; i < shi; ++i) {
        uint32_t v = 0, l = 0;
        int found = -1;
        while (found < 0) {
          if (l == HUFFREF_MAX_LEN || bit >= 8 * bytes) return H_ECORRUPT;
          v = (v << 1) | h_get_bit(blk, bit++);
          ++l;
          for (uint32_t sym = 0; sym < 256; ++sym)
            if (len[sym] == l && code[sym] == v) {
              found = (int)sym;
              break;
            }
        }
        out[i] = (uint8_t)found;
      }
    }
    if (h_div_up(bit, 32) * 4u != bytes) return H_ECORRUPT;
    pos += bytes;
  }
  *out_bytes = n;
  return H_OK;
}
