/*
 * lzref.h -- CPU oracle for chunked multi-byte LZSS (gpuLZ, ICS'23).
 *
 * TEST INFRASTRUCTURE ONLY.  This is the plain, slow, obviously-correct
 * definition that the CUDA path is checked against.  Only the test suite,
 * the smoke check and the CPU-baseline leg of the benchmark may call it.
 * It shares no code, header, table or helper with the CUDA library.
 *
 * What it computes (paper section 2.2, "LZSS", basic steps 1-6, restricted
 * to independent chunks as in section 3.3.1 and to S-byte symbols as in
 * section 3.2.3):
 *   per chunk, from coding position p = 0, take the longest run that the
 *   W previous symbols of the same chunk (the window) repeat from p (nearest
 *   offset on ties, match length <= offset, <= max_match, <= symbols left);
 *   emit a pointer (len, off) when len >= min_match, else a literal symbol;
 *   one flag bit per token (1 = pointer, 0 = literal).
 *
 * Stream layout "GLZ1" (the paper prints no container; this is the
 * reading used by both sides, all integers little-endian):
 *   [0,32)   header: "GLZ1", u8 version=1, u8 S, u8 offB, u8 m, u8 M,
 *            3 zero bytes, u32 chunk_bytes, u32 W, u32 n_chunks, u64 n_bytes
 *   table    n_chunks x {u32 n_tokens, u32 payload_bytes}
 *   index    ceil(n_chunks/64) x u64: byte offset of the record of chunk
 *            64*j, relative to the start of the records region
 *   records  per chunk in order: ceil(n_tokens/8) flag bytes (token t is
 *            bit t&7, LSB first, of byte t>>3; pad bits 0), then the
 *            payload: a literal is its S bytes, a pointer is u8 len then
 *            (off-1) as u8 (offB=1, W<=256) or u16 (offB=2).
 *
 * Return codes: 0 ok, 1 invalid argument, 2 output buffer too small,
 * 3 corrupt stream.
 */
#ifndef LZREF_H
#define LZREF_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* 0 if (S, C, W, m, M) is a valid parameter set, else 1. */
int lzref_check_params(uint32_t S, uint32_t C, uint32_t W, uint32_t m,
                       uint32_t M);

/* Largest stream compress can produce for n bytes (any version; a tail of
 * n % S bytes adds itself); 0 for invalid params. */
uint64_t lzref_bound(uint64_t n, uint32_t S, uint32_t C, uint32_t W,
                     uint32_t m, uint32_t M);

/* Longest match at symbol p of a chunk of k symbols (section 2.2 step 2).
 * Writes the length (0 if none) and the nearest offset achieving it. */
void lzref_longest_match(const uint8_t *chunk, uint32_t k, uint32_t p,
                         uint32_t S, uint32_t W, uint32_t M,
                         uint32_t *len, uint32_t *off);

/* The paper's matcher at symbol p (section 3.3.2, its four matching
 * steps): a forward scan of the window with a search pointer that is never
 * moved back, see lzref.c.  Writes the length of the first longest run it
 * meets (0 if none) and that run's offset.  Length <= offset, <= M and <=
 * k - p, as for lzref_longest_match, which it never exceeds. */
void lzref_paper_match(const uint8_t *chunk, uint32_t k, uint32_t p,
                       uint32_t S, uint32_t W, uint32_t M, uint32_t *len,
                       uint32_t *off);

/* The exact longest match with overlapping allowed (length bounded by M
 * and k - p only, not by the offset); nearest offset on ties. */
void lzref_longest_match_overlap(const uint8_t *chunk, uint32_t k, uint32_t p,
                                 uint32_t S, uint32_t W, uint32_t M,
                                 uint32_t *len, uint32_t *off);

/* Matchers of the greedy parse. */
#define LZREF_MATCH_EXACT 0u   /* lzref_longest_match (the definition) */
#define LZREF_MATCH_PAPER 1u   /* lzref_paper_match (the paper's method) */
#define LZREF_MATCH_OVERLAP 2u /* lzref_longest_match_overlap; version 2 */

/* Greedy parse of one chunk.  tok_len[t] = symbols covered by token t,
 * tok_off[t] = pointer offset in symbols (0 for a literal).  Arrays must
 * hold k entries.  Returns the number of tokens. */
uint32_t lzref_parse_chunk(const uint8_t *chunk, uint32_t k, uint32_t S,
                           uint32_t W, uint32_t m, uint32_t M,
                           uint32_t *tok_len, uint32_t *tok_off);

uint32_t lzref_parse_chunk_mode(const uint8_t *chunk, uint32_t k, uint32_t S,
                                uint32_t W, uint32_t m, uint32_t M,
                                uint32_t mode, uint32_t *tok_len,
                                uint32_t *tok_off);

int lzref_compress(const uint8_t *in, uint64_t n, uint32_t S, uint32_t C,
                   uint32_t W, uint32_t m, uint32_t M, uint8_t *out,
                   uint64_t cap, uint64_t *out_bytes);

/* lzref_compress with the matcher `mode` (LZREF_MATCH_*); the stream
 * layout does not depend on it. */
int lzref_compress_mode(const uint8_t *in, uint64_t n, uint32_t S, uint32_t C,
                        uint32_t W, uint32_t m, uint32_t M, uint32_t mode,
                        uint8_t *out, uint64_t cap, uint64_t *out_bytes);

/* lzref_compress_mode writing stream version `version`:
 *   1  the layout above;
 *   2  the same layout (version byte 2) in which a chunk whose coded record
 *      (flag bytes + payload) would be at least as large as the chunk
 *      itself is stored instead: table entry {0, chunk bytes}, record =
 *      the chunk's bytes (no flags).  A coded chunk always has >= 1 token,
 *      so a token count of 0 marks a stored chunk unambiguously.  n need
 *      not be a multiple of S: the last chunk's 1..S-1 bytes past its last
 *      whole symbol follow its payload as they are (counted in
 *      payload_bytes), and a chunk with no whole symbol is stored.  Header
 *      byte 9 is 1 when the stream was parsed with LZREF_MATCH_OVERLAP
 *      (pointers may be longer than their offset), else 0; the decoders
 *      reject a pointer longer than its offset in a stream without it.
 * The decoder reads both versions. */
int lzref_compress_v(const uint8_t *in, uint64_t n, uint32_t S, uint32_t C,
                     uint32_t W, uint32_t m, uint32_t M, uint32_t mode,
                     uint32_t version, uint8_t *out, uint64_t cap,
                     uint64_t *out_bytes);

/* Reads n_bytes from a header (version 1 or 2); 0 ok, 3 corrupt. */
int lzref_decompressed_size(const uint8_t *in, uint64_t in_bytes,
                            uint64_t *n);

int lzref_decompress(const uint8_t *in, uint64_t in_bytes, uint8_t *out,
                     uint64_t cap, uint64_t *out_bytes);

#ifdef __cplusplus
}
#endif
#endif
