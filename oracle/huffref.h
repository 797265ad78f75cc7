/*
 * huffref.h -- CPU oracle for the Huffman stage that follows LZSS in the
 * paper's use case (section 4.5: cuSZ's Huffman encoding after gpuLZ).
 *
 * TEST INFRASTRUCTURE ONLY, like lzref.h: only the test suite, the smoke
 * check and the CPU-baseline leg of the benchmark may call it, and it shares
 * nothing with the CUDA library.
 *
 * The paper names the stage (Huffman encoding of the bytes gpuLZ produces)
 * but prints no format, so this stage's definition is ours:
 *   - alphabet: the 256 byte values of the input;
 *   - code lengths: an optimal prefix code under a maximum length of
 *     HUFFREF_MAX_LEN bits, found by package-merge (Larmore and Hirschberg,
 *     1990) with the tie rules in huffref.c; one symbol present gets
 *     length 1, none gets no code;
 *   - codes: canonical (symbols in order of (length, value) get
 *     consecutive codes, shifted left when the length grows);
 *   - stream "GHF1" (integers little-endian):
 *       [0,16)    "GHF1", u32 block bytes (HUFFREF_BLOCK), u64 n_bytes
 *       [16,272)  256 x u8 code length of each byte value
 *       table     n_blocks x u64: end of each block's bit string, in bytes
 *                 from the start of `bits` (block b spans [end[b-1], end[b]),
 *                 end[-1] = 0)
 *       subs      n_blocks x 32 x u32: bit offset, inside its block's bit
 *                 string, of each of the block's 32 sub-blocks of
 *                 HUFFREF_SUB input bytes (offset 0 first; sub-blocks past
 *                 the input's end repeat the end offset)
 *       bits      the blocks' bit strings, each a whole number of u32 words:
 *                 bit i of a block is bit 31 - (i % 32) of its word i / 32
 *                 (codes most significant bit first), padding bits 0.
 * Return codes: 0 ok, 1 invalid argument, 2 output too small, 3 corrupt.
 */
#ifndef HUFFREF_H
#define HUFFREF_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define HUFFREF_MAX_LEN 12u
#define HUFFREF_BLOCK 32768u
#define HUFFREF_SUB 1024u

/* Code lengths (0 = absent) of an optimal prefix code for the counts
 * hist[256] with no length above max_len (1..16). */
void huffref_lengths(const uint64_t *hist, uint32_t max_len, uint8_t *len);

/* Canonical codes for the lengths len[256] (code[s] holds len[s] bits). */
void huffref_codes(const uint8_t *len, uint32_t *code);

/* Largest stream huffref_compress can produce for n bytes. */
uint64_t huffref_bound(uint64_t n);

int huffref_compress(const uint8_t *in, uint64_t n, uint8_t *out,
                     uint64_t cap, uint64_t *out_bytes);

int huffref_decompressed_size(const uint8_t *in, uint64_t in_bytes,
                              uint64_t *n);

int huffref_decompress(const uint8_t *in, uint64_t in_bytes, uint8_t *out,
                       uint64_t cap, uint64_t *out_bytes);

#ifdef __cplusplus
}
#endif
#endif
