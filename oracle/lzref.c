/*
 * lzref.c -- CPU oracle for chunked multi-byte LZSS.  TEST INFRASTRUCTURE
 * ONLY (see lzref.h): the tests, the smoke check and the CPU-baseline leg
 * of the benchmark call it; the product never does.
 *
 * Everything here is the plain definition, written for a reader to check
 * against the paper by eye: no blocking, no hashing, no early exits that
 * the definition does not have.  Cost is O(k * W * len) per chunk.
 */
#include "lzref.h"

#include <stdlib.h>
#include <string.h>

enum { REF_OK = 0, REF_EINVAL = 1, REF_ESMALL = 2, REF_ECORRUPT = 3 };

#define REF_HEADER_BYTES 32u
#define REF_TABLE_ENTRY 8u
#define REF_INDEX_STRIDE 64u

/* Parameter set (one reading of section 3.2.3 and Table 1's grid):
 *   S (symbol bytes) in {1,2,4}; C (chunk bytes) a multiple of 16 in
 *   [16, 32768]; W (window, symbols) in [1, 1024]; 1 <= m <= M <= 255,
 *   M fitting the one-byte length field of section 3.3.2. */
int lzref_check_params(uint32_t S, uint32_t C, uint32_t W, uint32_t m,
                       uint32_t M) {
  if (S != 1 && S != 2 && S != 4) return REF_EINVAL;
  if (C < 16 || C > 32768 || C % 16 != 0) return REF_EINVAL;
  if (W < 1 || W > 1024) return REF_EINVAL;
  if (m < 1 || m > M || M > 255) return REF_EINVAL;
  return REF_OK;
}

/* Offset field width: one byte while every offset-1 fits in 8 bits. */
static uint32_t ref_off_bytes(uint32_t W) { return W <= 256 ? 1u : 2u; }

static uint64_t ref_div_up(uint64_t a, uint64_t b) { return (a + b - 1) / b; }

/* Worst-case record of a chunk of k symbols: flags for k tokens plus the
 * largest payload a parse can have.  A parse with `lit` literal symbols
 * and the rest covered by pointers of >= m symbols has payload
 * S*lit + (1+offB)*floor((k-lit)/m); its maximum over lit is
 * S*k + max(0, 1+offB-S*m)*floor(k/m). */
static uint64_t ref_record_bound(uint64_t k, uint32_t S, uint32_t offB,
                                 uint32_t m) {
  uint64_t extra = (1u + offB > S * m) ? (1u + offB - S * m) : 0u;
  return ref_div_up(k, 8) + (uint64_t)S * k + extra * (k / m);
}

uint64_t lzref_bound(uint64_t n, uint32_t S, uint32_t C, uint32_t W,
                     uint32_t m, uint32_t M) {
  if (lzref_check_params(S, C, W, m, M) != REF_OK) return 0;
  uint64_t nc = ref_div_up(n, C);
  uint64_t total = REF_HEADER_BYTES + REF_TABLE_ENTRY * nc +
                   8u * ref_div_up(nc, REF_INDEX_STRIDE);
  uint32_t offB = ref_off_bytes(W);
  for (uint64_t c = 0; c < nc; ++c) {
    uint64_t bytes = (c + 1 < nc) ? C : n - c * (uint64_t)C;
    total += ref_record_bound(bytes / S, S, offB, m) + bytes % S;
  }
  return total;
}

/* Symbols i and j of a chunk are equal iff their S bytes are equal. */
static int ref_sym_eq(const uint8_t *chunk, uint32_t S, uint32_t i,
                      uint32_t j) {
  return memcmp(chunk + (size_t)i * S, chunk + (size_t)j * S, S) == 0;
}

/* Section 2.2 step 2, over S-byte symbols (section 3.2.3):
 * for every offset d = 1 .. min(W, p) extend the match symbol by symbol
 * while it stays within min(M, d, k-p) symbols (a pointer may not run into
 * the coding position, section 3.3.2); keep the first d that reaches the
 * largest length, which is the nearest one. */
void lzref_longest_match(const uint8_t *chunk, uint32_t k, uint32_t p,
                         uint32_t S, uint32_t W, uint32_t M, uint32_t *len,
                         uint32_t *off) {
  uint32_t best = 0, best_d = 0;
  uint32_t dmax = W < p ? W : p;
  for (uint32_t d = 1; d <= dmax; ++d) {
    uint32_t cap = M;
    if (d < cap) cap = d;
    if (k - p < cap) cap = k - p;
    uint32_t l = 0;
    while (l < cap && ref_sym_eq(chunk, S, p + l, p - d + l)) ++l;
    if (l > best) {
      best = l;
      best_d = d;
    }
  }
  *len = best;
  *off = best_d;
}

/* The paper's own matcher (section 3.3.2, the four steps of its matching
 * method), over S-byte symbols, stated run by run.  The scan goes through
 * the window from its far end, p - min(W, p), towards the coding position
 * p:
 *   1. the next window symbol equal to the one at p starts a run (no other
 *      symbol can start one);
 *   2. the run is measured: the number of symbols that agree with the
 *      look-ahead from p, stopping at a mismatch, when the run would reach
 *      p (so length <= offset) or at the end of the look-ahead;
 *   3. a run strictly longer than the longest so far replaces it, with
 *      offset p - (run start);
 *   4. a run that reached p or the look-ahead end ends the scan; otherwise
 *      the scan resumes just after the symbol that broke the run -- that
 *      symbol itself is never tried as a run start, and the scan never
 *      goes back into the run, which is why the method can miss the
 *      longest match.
 * Readings where the paper is silent: the look-ahead ends at the chunk end
 * or M symbols after p, whichever comes first (the length field is one
 * byte); the run that ends the scan is compared like any other (otherwise
 * a run that reaches p would never count).  Ties keep the first run found,
 * i.e. the farthest offset. */
void lzref_paper_match(const uint8_t *chunk, uint32_t k, uint32_t p,
                       uint32_t S, uint32_t W, uint32_t M, uint32_t *len,
                       uint32_t *off) {
  const uint32_t end = (k - p < M) ? k : p + M;  /* look-ahead end */
  uint32_t best = 0, best_off = 0;
  uint32_t w = p > W ? p - W : 0;
  while (w < p) {
    if (!ref_sym_eq(chunk, S, w, p)) { /* step 1: not a run start */
      ++w;
      continue;
    }
    uint32_t l = 0; /* step 2 */
    while (w + l < p && p + l < end && ref_sym_eq(chunk, S, w + l, p + l)) ++l;
    if (l > best) { /* step 3 */
      best = l;
      best_off = p - w;
    }
    if (w + l == p || p + l == end) break; /* step 4 */
    w += l + 1;
  }
  *len = best;
  *off = best_off;
}

/* The exact longest match when a match may overlap the look-ahead (stream
 * version 2's overlap mode): as lzref_longest_match, but a match may run on
 * into the symbols it produces, so its length is bounded by M and by the
 * symbols left in the chunk only (the classic LZ77 reading; section 3.3.2
 * forbids it for the paper's own format).  Nearest offset on ties. */
void lzref_longest_match_overlap(const uint8_t *chunk, uint32_t k, uint32_t p,
                                 uint32_t S, uint32_t W, uint32_t M,
                                 uint32_t *len, uint32_t *off) {
  uint32_t best = 0, best_d = 0;
  uint32_t dmax = W < p ? W : p;
  for (uint32_t d = 1; d <= dmax; ++d) {
    uint32_t cap = M;
    if (k - p < cap) cap = k - p;
    uint32_t l = 0;
    while (l < cap && ref_sym_eq(chunk, S, p + l, p - d + l)) ++l;
    if (l > best) {
      best = l;
      best_d = d;
    }
  }
  *len = best;
  *off = best_d;
}

typedef void (*ref_matcher)(const uint8_t *, uint32_t, uint32_t, uint32_t,
                            uint32_t, uint32_t, uint32_t *, uint32_t *);

static ref_matcher ref_matcher_of(uint32_t mode) {
  if (mode == LZREF_MATCH_PAPER) return lzref_paper_match;
  if (mode == LZREF_MATCH_OVERLAP) return lzref_longest_match_overlap;
  return lzref_longest_match;
}

/* Section 2.2 steps 1, 3, 4, 6: greedy parse from the chunk start. */
uint32_t lzref_parse_chunk(const uint8_t *chunk, uint32_t k, uint32_t S,
                           uint32_t W, uint32_t m, uint32_t M,
                           uint32_t *tok_len, uint32_t *tok_off) {
  return lzref_parse_chunk_mode(chunk, k, S, W, m, M, LZREF_MATCH_EXACT,
                                tok_len, tok_off);
}

uint32_t lzref_parse_chunk_mode(const uint8_t *chunk, uint32_t k, uint32_t S,
                                uint32_t W, uint32_t m, uint32_t M,
                                uint32_t mode, uint32_t *tok_len,
                                uint32_t *tok_off) {
  ref_matcher match = ref_matcher_of(mode);
  uint32_t p = 0, t = 0;
  while (p < k) {
    uint32_t len, off;
    match(chunk, k, p, S, W, M, &len, &off);
    if (len >= m) {
      tok_len[t] = len;
      tok_off[t] = off;
      p += len;
    } else {
      tok_len[t] = 1;
      tok_off[t] = 0;
      p += 1;
    }
    ++t;
  }
  return t;
}

static void ref_put_u32(uint8_t *dst, uint32_t v) {
  for (int i = 0; i < 4; ++i) dst[i] = (uint8_t)(v >> (8 * i));
}
static void ref_put_u64(uint8_t *dst, uint64_t v) {
  for (int i = 0; i < 8; ++i) dst[i] = (uint8_t)(v >> (8 * i));
}
static uint32_t ref_get_u32(const uint8_t *src) {
  uint32_t v = 0;
  for (int i = 0; i < 4; ++i) v |= (uint32_t)src[i] << (8 * i);
  return v;
}
static uint64_t ref_get_u64(const uint8_t *src) {
  uint64_t v = 0;
  for (int i = 0; i < 8; ++i) v |= (uint64_t)src[i] << (8 * i);
  return v;
}

int lzref_compress(const uint8_t *in, uint64_t n, uint32_t S, uint32_t C,
                   uint32_t W, uint32_t m, uint32_t M, uint8_t *out,
                   uint64_t cap, uint64_t *out_bytes) {
  return lzref_compress_mode(in, n, S, C, W, m, M, LZREF_MATCH_EXACT, out, cap,
                             out_bytes);
}

int lzref_compress_mode(const uint8_t *in, uint64_t n, uint32_t S, uint32_t C,
                        uint32_t W, uint32_t m, uint32_t M, uint32_t mode,
                        uint8_t *out, uint64_t cap, uint64_t *out_bytes) {
  return lzref_compress_v(in, n, S, C, W, m, M, mode, 1, out, cap, out_bytes);
}

int lzref_compress_v(const uint8_t *in, uint64_t n, uint32_t S, uint32_t C,
                     uint32_t W, uint32_t m, uint32_t M, uint32_t mode,
                     uint32_t version, uint8_t *out, uint64_t cap,
                     uint64_t *out_bytes) {
  if (lzref_check_params(S, C, W, m, M) != REF_OK) return REF_EINVAL;
  if (mode != LZREF_MATCH_EXACT && mode != LZREF_MATCH_PAPER &&
      mode != LZREF_MATCH_OVERLAP)
    return REF_EINVAL;
  if (version != 1 && version != 2) return REF_EINVAL;
  if (mode == LZREF_MATCH_OVERLAP && version != 2) return REF_EINVAL;
  if (version == 1 && n % S != 0) return REF_EINVAL;
  uint64_t nc = ref_div_up(n, C);
  if (nc > 0xFFFFFFFFull) return REF_EINVAL;
  uint32_t offB = ref_off_bytes(W);
  uint64_t n_index = ref_div_up(nc, REF_INDEX_STRIDE);
  uint64_t table_at = REF_HEADER_BYTES;
  uint64_t index_at = table_at + REF_TABLE_ENTRY * nc;
  uint64_t records_at = index_at + 8u * n_index;
  if (cap < records_at) return REF_ESMALL;

  memset(out, 0, (size_t)records_at);
  memcpy(out, "GLZ1", 4);
  out[4] = (uint8_t)version;
  out[9] = mode == LZREF_MATCH_OVERLAP ? 1u : 0u; /* overlap flag (version 2) */
  out[5] = (uint8_t)S;
  out[6] = (uint8_t)offB;
  out[7] = (uint8_t)m;
  out[8] = (uint8_t)M;
  ref_put_u32(out + 12, C);
  ref_put_u32(out + 16, W);
  ref_put_u32(out + 20, (uint32_t)nc);
  ref_put_u64(out + 24, n);

  uint32_t kmax = C / S;
  uint32_t *tok_len = (uint32_t *)malloc(sizeof(uint32_t) * kmax);
  uint32_t *tok_off = (uint32_t *)malloc(sizeof(uint32_t) * kmax);
  if (!tok_len || !tok_off) {
    free(tok_len);
    free(tok_off);
    return REF_EINVAL;
  }

  uint64_t pos = records_at; /* write cursor (absolute) */
  int rc = REF_OK;
  for (uint64_t c = 0; c < nc; ++c) {
    const uint8_t *chunk = in + c * (uint64_t)C;
    uint64_t bytes = (c + 1 < nc) ? C : n - c * (uint64_t)C;
    uint32_t k = (uint32_t)(bytes / S);
    uint32_t ntok =
        lzref_parse_chunk_mode(chunk, k, S, W, m, M, mode, tok_len, tok_off);

    if (c % REF_INDEX_STRIDE == 0)
      ref_put_u64(out + index_at + 8u * (c / REF_INDEX_STRIDE),
                  pos - records_at);

    uint32_t flag_bytes = (ntok + 7) / 8;
    uint64_t payload = 0;
    for (uint32_t t = 0; t < ntok; ++t)
      payload += tok_off[t] ? 1u + offB : S;
    /* version 2: the 1..S-1 bytes past the last whole symbol (last chunk
     * only) follow the tokens, as they are */
    uint32_t tail = (uint32_t)(bytes - (uint64_t)k * S);
    payload += tail;

    /* version 2: a chunk whose coded record would not be smaller than its
     * bytes is stored as they are, marked by a token count of 0 */
    if (version == 2 && flag_bytes + payload >= bytes) {
      ref_put_u32(out + table_at + REF_TABLE_ENTRY * c, 0);
      ref_put_u32(out + table_at + REF_TABLE_ENTRY * c + 4, (uint32_t)bytes);
      if (pos + bytes > cap) {
        rc = REF_ESMALL;
        break;
      }
      memcpy(out + pos, chunk, (size_t)bytes);
      pos += bytes;
      continue;
    }
    ref_put_u32(out + table_at + REF_TABLE_ENTRY * c, ntok);
    ref_put_u32(out + table_at + REF_TABLE_ENTRY * c + 4, (uint32_t)payload);

    if (pos + flag_bytes + payload > cap) {
      rc = REF_ESMALL;
      break;
    }
    uint8_t *flags = out + pos;
    memset(flags, 0, flag_bytes);
    uint8_t *pay = flags + flag_bytes;
    uint32_t p = 0; /* symbol cursor inside the chunk */
    for (uint32_t t = 0; t < ntok; ++t) {
      if (tok_off[t]) {
        flags[t >> 3] |= (uint8_t)(1u << (t & 7));
        *pay++ = (uint8_t)tok_len[t];
        uint32_t stored = tok_off[t] - 1;
        *pay++ = (uint8_t)(stored & 0xFF);
        if (offB == 2) *pay++ = (uint8_t)(stored >> 8);
      } else {
        memcpy(pay, chunk + (size_t)p * S, S);
        pay += S;
      }
      p += tok_len[t];
    }
    memcpy(pay, chunk + (size_t)k * S, tail);
    pos += flag_bytes + payload;
  }
  free(tok_len);
  free(tok_off);
  if (rc != REF_OK) return rc;
  *out_bytes = pos;
  return REF_OK;
}

/* Header checks shared by both decoder entry points. */
static int ref_read_header(const uint8_t *in, uint64_t in_bytes,
                           uint32_t *S, uint32_t *offB, uint32_t *C,
                           uint32_t *W, uint32_t *m, uint32_t *M,
                           uint64_t *nc, uint64_t *n) {
  if (in_bytes < REF_HEADER_BYTES) return REF_ECORRUPT;
  if (memcmp(in, "GLZ1", 4) != 0 || (in[4] != 1 && in[4] != 2)) return REF_ECORRUPT;
  if (in[9] > (in[4] == 2 ? 1 : 0) || in[10] || in[11]) return REF_ECORRUPT;
  *S = in[5];
  *offB = in[6];
  *m = in[7];
  *M = in[8];
  *C = ref_get_u32(in + 12);
  *W = ref_get_u32(in + 16);
  *nc = ref_get_u32(in + 20);
  *n = ref_get_u64(in + 24);
  if (lzref_check_params(*S, *C, *W, *m, *M) != REF_OK) return REF_ECORRUPT;
  if (*offB != ref_off_bytes(*W)) return REF_ECORRUPT;
  if (in[4] == 1 && *n % *S != 0) return REF_ECORRUPT; /* tails: version 2 */
  if (*nc != ref_div_up(*n, *C)) return REF_ECORRUPT;
  return REF_OK;
}

int lzref_decompressed_size(const uint8_t *in, uint64_t in_bytes,
                            uint64_t *n) {
  uint32_t S, offB, C, W, m, M;
  uint64_t nc;
  int rc = ref_read_header(in, in_bytes, &S, &offB, &C, &W, &m, &M, &nc, n);
  return rc;
}

/* Inverse of lzref_compress.  Pointers are copied symbol by symbol in
 * token order, so a source that is itself pointer output is already in
 * place when it is read. */
int lzref_decompress(const uint8_t *in, uint64_t in_bytes, uint8_t *out,
                     uint64_t cap, uint64_t *out_bytes) {
  uint32_t S, offB, C, W, m, M;
  uint64_t nc, n;
  int rc = ref_read_header(in, in_bytes, &S, &offB, &C, &W, &m, &M, &nc, &n);
  if (rc != REF_OK) return rc;
  uint64_t n_index = ref_div_up(nc, REF_INDEX_STRIDE);
  uint64_t table_at = REF_HEADER_BYTES;
  uint64_t index_at = table_at + REF_TABLE_ENTRY * nc;
  uint64_t records_at = index_at + 8u * n_index;
  if (in_bytes < records_at) return REF_ECORRUPT;
  if (cap < n) return REF_ESMALL;

  uint64_t pos = records_at;
  for (uint64_t c = 0; c < nc; ++c) {
    if (c % REF_INDEX_STRIDE == 0 &&
        ref_get_u64(in + index_at + 8u * (c / REF_INDEX_STRIDE)) !=
            pos - records_at)
      return REF_ECORRUPT;
    uint32_t ntok = ref_get_u32(in + table_at + REF_TABLE_ENTRY * c);
    uint32_t payload = ref_get_u32(in + table_at + REF_TABLE_ENTRY * c + 4);
    uint64_t flag_bytes = ((uint64_t)ntok + 7) / 8;
    if (pos + flag_bytes + payload > in_bytes) return REF_ECORRUPT;
    const uint8_t *flags = in + pos;
    const uint8_t *pay = flags + flag_bytes;
    const uint8_t *pay_end = pay + payload;
    uint8_t *dst = out + c * (uint64_t)C;
    uint64_t bytes = (c + 1 < nc) ? C : n - c * (uint64_t)C;
    uint32_t k = (uint32_t)(bytes / S);
    if (ntok == 0 && in[4] == 2) { /* a stored chunk: its bytes as they are */
      if (payload != bytes) return REF_ECORRUPT;
      memcpy(dst, pay, (size_t)bytes);
      pos += payload;
      continue;
    }
    uint32_t p = 0;
    for (uint32_t t = 0; t < ntok; ++t) {
      if (p >= k) return REF_ECORRUPT;
      if ((flags[t >> 3] >> (t & 7)) & 1u) {
        if (pay + 1 + offB > pay_end) return REF_ECORRUPT;
        uint32_t len = pay[0];
        uint32_t off = pay[1];
        if (offB == 2) off |= (uint32_t)pay[2] << 8;
        off += 1;
        pay += 1 + offB;
        /* an offset reaches at most W symbols back (section 2.2 sliding window)
         and never before the chunk start */
        if (len == 0 || off > p || off > W || len > k - p) return REF_ECORRUPT;
        if (len > off && !in[9]) return REF_ECORRUPT; /* overlap only if flagged */
        for (uint32_t i = 0; i < len; ++i)
          memcpy(dst + (size_t)(p + i) * S, dst + (size_t)(p + i - off) * S,
                 S);
        p += len;
      } else {
        if (pay + S > pay_end) return REF_ECORRUPT;
        memcpy(dst + (size_t)p * S, pay, S);
        pay += S;
        p += 1;
      }
    }
    uint32_t tail = (uint32_t)(bytes - (uint64_t)k * S);
    if (p != k || pay + tail != pay_end) return REF_ECORRUPT;
    memcpy(dst + (size_t)k * S, pay, tail);
    pos += flag_bytes + payload;
  }
  *out_bytes = n;
  return REF_OK;
}
