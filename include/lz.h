/*
 * lz.h -- C ABI of the GB300 (sm_103a) chunked multi-byte LZSS codec.
 *
 * Method: gpuLZ (ICS'23).  Compression is LZSS (section 2.2: greedy longest
 * match in a sliding window, pointer or literal, one flag bit per token)
 * over S-byte symbols (section 3.2.3), on independent chunks (section
 * 3.3.1), with the output offsets found by a two-pass prefix sum -- local
 * inside a chunk, then global over chunks (section 3.2.2) -- fused into the
 * matching/encoding kernel (section 3.3.2; the separate scan and deflate
 * kernels of sections 3.3.3/3.3.4 are folded into it).
 *
 * The parse is the exact greedy one: at each coding position the longest
 * match over offsets 1..min(W, p) (lengths bounded by M, by the offset and
 * by the symbols left in the chunk), the nearest offset on ties; a pointer
 * when its length is >= m, else a literal.  Output is byte-identical to the
 * CPU definition for the same parameters.
 *
 * Stream layout "GLZ1" (all integers little-endian; version 2, written by
 * lz_compress_ex on request, adds stored chunks and tail bytes, see
 * lz_options):
 *   header  32 B: "GLZ1", u8 version (1 or 2), u8 S, u8 offB, u8 m, u8 M,
 *           u8 overlap (version 2: 1 when pointers may be longer than their
 *           offset, else 0), 2 zero bytes, u32 chunk_bytes, u32 W,
 *           u32 n_chunks, u64 n_bytes
 *   table   n_chunks x {u32 n_tokens, u32 payload_bytes}
 *   index   ceil(n_chunks/64) x u64: offset of the record of chunk 64*j,
 *           relative to the start of the records region
 *   records per chunk: ceil(n_tokens/8) flag bytes (token t = bit t&7 of
 *           byte t>>3; 1 = pointer), then the payload: a literal is its S
 *           bytes, a pointer is u8 length then (offset-1) as u8 (offB = 1,
 *           W <= 256) or u16 (offB = 2).  Lengths and offsets count symbols.
 *
 * Conventions for every entry point below:
 *   - Pointers named d_* are device pointers (cudaMalloc, cudaMallocAsync,
 *     or a torch CUDA tensor's data pointer) on the context's device; the
 *     caller owns them.  h_* pointers are host pointers.
 *   - Calls are asynchronous on `stream` (a cudaStream_t; NULL = legacy
 *     default stream) and perform no host synchronisation, except
 *     lz_decompressed_size and lz_sync, which say so.
 *   - Argument errors are returned synchronously and nothing is enqueued.
 *   - Errors found on the device (output too small, corrupt stream,
 *     bounded device wait expired) are sticky in the context and returned
 *     (then cleared) by lz_sync.
 *   - A context serialises its work through one scratch area: calls that
 *     share a context must be ordered on one stream (use one context per
 *     concurrent stream).
 */
#ifndef GB300_LZ_H
#define GB300_LZ_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *lz_stream_t; /* same type as cudaStream_t */

typedef struct lz_params {
  uint32_t symbol_bytes; /* S: 1, 2 or 4 (section 3.2.3)                 */
  uint32_t chunk_bytes;  /* C: multiple of 16 in [16, 32768] (3.3.1)     */
  uint32_t window;       /* W: 1..1024 symbols (section 2.2, 3.2.3)      */
  uint32_t min_match;    /* m: 1..max_match (minimum pointer length)     */
  uint32_t max_match;    /* M: min_match..255 (one length byte, 3.3.2)   */
} lz_params;

/* Matcher of the greedy parse.  Both give streams of the same layout,
 * decoded by lz_decompress. */
typedef enum lz_match {
  LZ_MATCH_EXACT = 0, /* longest match, nearest offset on ties (section 2.2
                         step 2, the definition; what lz_compress uses)   */
  LZ_MATCH_PAPER = 1,  /* the paper's own matcher (section 3.3.2, the four
                         steps of its matching method): a forward scan of
                         the window from its far end whose search pointer
                         never moves back, keeping the first run of the
                         greatest length; it can miss the longest match */
  LZ_MATCH_OVERLAP = 2 /* the exact longest match when a match may run on
                         into the symbols it produces (length bounded by M
                         and the chunk end, not by the offset; classic LZ77,
                         which section 3.3.2 does not use); stream version 2
                         only, recorded in header byte 9 */
} lz_match;

typedef enum lz_status {
  LZ_OK = 0,
  LZ_ERR_INVALID_ARG = 1,      /* bad pointer, size or parameter          */
  LZ_ERR_BUFFER_TOO_SMALL = 2, /* output capacity below what is needed    */
  LZ_ERR_CORRUPT = 3,          /* input is not a well-formed GLZ1 stream  */
  LZ_ERR_NOMEM = 4,            /* context scratch allocation failed       */
  LZ_ERR_CUDA = 5,             /* CUDA runtime error (launch, copy, ...)  */
  LZ_ERR_TIMEOUT = 6,          /* a bounded device-side wait gave up      */
  LZ_ERR_INTERNAL = 7          /* a device-side consistency check failed
                                  (a bug in this library; output invalid) */
} lz_status;

typedef struct lz_ctx lz_ctx;

/* Create a context on `device` (cudaSetDevice is called on it).  The
 * context owns a small device scratch area (chunk status words for the
 * global scan, a work counter, the sticky error word).  Returns
 * LZ_ERR_INVALID_ARG for a null ctx or bad device, LZ_ERR_NOMEM or
 * LZ_ERR_CUDA on allocation failure. */
lz_status lz_create(lz_ctx **ctx, int device);

/* Free a context (synchronises the device first).  NULL is ignored. */
void lz_destroy(lz_ctx *ctx);

/* Human-readable name of a status code (static string). */
const char *lz_status_string(lz_status s);

/* LZ_OK if *p is a valid parameter set, else LZ_ERR_INVALID_ARG. */
lz_status lz_check_params(const lz_params *p);

/* Pure host function: the largest stream lz_compress can produce for
 * n_bytes of input with parameters *p, i.e. header + table + index + per
 * chunk ceil(k/8) + S*k + max(0, 1+offB-S*m)*floor(k/m) (k = symbols in the
 * chunk).  Returns 0 if *p is invalid. */
uint64_t lz_compressed_bound(uint64_t n_bytes, const lz_params *p);

/* Compress n_bytes at d_in (n_bytes % S == 0; n_bytes == 0 allowed) into
 * d_out (capacity out_cap bytes) and store the stream size in *d_out_bytes
 * (a device uint64, 8-byte aligned).  One kernel launch (plus a scratch
 * clear); d_in is staged with TMA bulk copies when it is 16-byte aligned.
 * Returns LZ_ERR_BUFFER_TOO_SMALL synchronously when out_cap cannot even
 * hold header + table + index; if the records do not fit, the stream is
 * incomplete, *d_out_bytes still receives the size that was needed and
 * lz_sync reports LZ_ERR_BUFFER_TOO_SMALL.  Capacity
 * lz_compressed_bound(n_bytes, p) always suffices.  LZ_ERR_INVALID_ARG
 * beyond 2^32 - 2^20 - 1 chunks (the work counter is 32 bits wide). */
lz_status lz_compress(lz_ctx *ctx, const void *d_in, uint64_t n_bytes,
                      const lz_params *p, void *d_out, uint64_t out_cap,
                      uint64_t *d_out_bytes, lz_stream_t stream);

/* Options of lz_compress_ex.  A zero-initialised struct means
 * LZ_MATCH_EXACT and stream version 1, i.e. exactly lz_compress. */
typedef struct lz_options {
  uint32_t match;   /* lz_match                                          */
  uint32_t version; /* stream version written: 0 or 1 = version 1 above;
                       2 = the same layout with version byte 2, in which
                       (a) a chunk whose coded record (flag bytes +
                       payload) would not be smaller than the chunk is
                       stored as it is: table entry {0, chunk bytes},
                       record = the chunk's bytes, no flags (a coded
                       chunk has >= 1 token, so 0 marks it); and (b)
                       n_bytes need not be a multiple of S: the last
                       chunk's 1..S-1 bytes after its last whole symbol
                       follow its tokens as they are, counted in its
                       payload_bytes.  lz_decompress reads both.       */
  uint32_t warps_per_block; /* compression launch shape: warps per block
                       (one chunk per warp at a time): 1, 2, 4 or 8;
                       0 = the library's choice, the one that keeps the
                       most warps resident.  It changes how chunks are
                       spread over the GPU, never the stream.          */
} lz_options;

/* lz_compress with options (opt may be NULL: the defaults).
 * opt->match = LZ_MATCH_PAPER parses with the paper's matcher (section
 * 3.3.2): at coding position p the scan runs from max(0, p - W); a run
 * that ends at a mismatch is kept if strictly longer than the best so far,
 * and the scan resumes at the symbol after the one that broke it; the scan
 * ends when a run reaches p or the end of the look-ahead, min(k, p + M)
 * symbols; the parse takes a pointer when the kept run has >= m symbols.
 * Positions without any match of >= m symbols are literals under both
 * matchers, and the stream header does not record the matcher.
 * LZ_ERR_INVALID_ARG for an unknown matcher or version, for LZ_MATCH_OVERLAP
 * in version 1, or for n_bytes % S != 0 in version 1; everything else as
 * for lz_compress
 * (lz_compressed_bound covers both versions, a tail included). */
lz_status lz_compress_ex(lz_ctx *ctx, const void *d_in, uint64_t n_bytes,
                         const lz_params *p, const lz_options *opt, void *d_out,
                         uint64_t out_cap, uint64_t *d_out_bytes, lz_stream_t stream);

/* Compression from host memory to host memory: the same stream as
 * lz_compress of the same bytes, for callers whose data lives on the host.
 * h_in (n_bytes) and h_out (capacity out_cap) are host buffers.  The input
 * is copied to the device in pieces of whole index superblocks (64 chunks;
 * about 64 MiB a piece, smaller at both ends: 8, 16, 32 MiB first and
 * last), and each piece is compressed by a launch over its
 * own chunks as soon as it has arrived, while the next piece is copied:
 * chunks are independent (section 3.3.1) and the look-back of a piece's
 * first chunks reaches into the pieces before it, which are complete.
 * The stream is built in device memory.  When h_out is pinned
 * (cudaHostAlloc / cudaHostRegister), the records of each piece are copied
 * to it as soon as the piece is done (the host reads where they end), on a
 * third stream, while later pieces are copied in and compressed: the host
 * link carries both directions at once; the header, table and index follow
 * at the end.  Pageable h_out gets the stream in one copy at the end.
 * Pinned h_in lets the copies overlap the compression.  The context holds
 * device memory for the input and the stream between calls.  The call is
 * synchronous: it starts after the work already enqueued on `stream` and
 * returns when h_out holds the stream and *h_out_bytes (host) its size.
 * Device errors of this call are returned by it (and cleared), not left for
 * lz_sync.  LZ_ERR_BUFFER_TOO_SMALL when out_cap is below the stream size
 * (then *h_out_bytes is the size needed and h_out is incomplete);
 * LZ_ERR_NOMEM when the device memory cannot be had; argument errors as
 * for lz_compress (stream version 1, exact matcher). */
lz_status lz_compress_host(lz_ctx *ctx, const void *h_in, uint64_t n_bytes, const lz_params *p,
                           void *h_out, uint64_t out_cap, uint64_t *h_out_bytes,
                           lz_stream_t stream);

/* Read and validate the header of the stream at d_in (in_bytes long) and
 * return its decompressed size in *h_n.  Synchronises `stream` (it copies
 * the 32-byte header to the host).  LZ_ERR_CORRUPT for a bad header. */
lz_status lz_decompressed_size(const void *d_in, uint64_t in_bytes,
                               uint64_t *h_n, lz_stream_t stream);

/* Decompress the stream at d_in (in_bytes long) into d_out (capacity
 * out_cap bytes) and store the output size in *d_out_bytes (device
 * uint64).  Nothing about the stream needs to be known on the host: the
 * kernel reads the header, table and index itself.  Structural errors
 * (bad header, truncated record, offset before the chunk start or beyond
 * the window, token overrun, payload size mismatch, inconsistent index)
 * are reported as LZ_ERR_CORRUPT and out_cap < n_bytes as
 * LZ_ERR_BUFFER_TOO_SMALL, both by lz_sync.  in_bytes < 32 is rejected
 * synchronously with LZ_ERR_CORRUPT. */
lz_status lz_decompress(lz_ctx *ctx, const void *d_in, uint64_t in_bytes,
                        void *d_out, uint64_t out_cap, uint64_t *d_out_bytes,
                        lz_stream_t stream);

/* Compression for callers that cannot allocate device memory (no paper
 * counterpart; an addition of this library).  Same stream as lz_compress,
 * on the current device, with no context: the scratch is a fixed device
 * array inside the library (512 KiB + 16 B, held by every GPU that loads
 * the library until the process exits), so the call allocates nothing and
 * n_bytes may span at most 65536 chunks (LZ_ERR_INVALID_ARG beyond that).
 * The caller passes inputs and outputs as for lz_compress.  Device-side
 * outcomes are reported through *d_out_bytes: a value <= out_cap is the
 * stream size (success); a value > out_cap is the size that was needed
 * (output too small, stream incomplete); 0 means a device-side check failed.
 * Every call shares the fixed array, so calls whose work overlaps on the GPU
 * (other streams, other threads) race and must not be issued; calls ordered
 * on one stream are fine.  The first call on a device looks up the array's
 * device address (and launch limits); make that first call before any
 * stream capture.  Under CUDA's lazy module loading (the default) the first
 * launch of each kernel variant loads its code onto the device, which takes
 * device memory: before entering a region where nothing may be allocated,
 * make one call for every symbol size and window class it will use (window
 * classes: W <= 32, <= 64, <= 128, <= 256, <= 512, <= 1024), plus one with
 * n_bytes = 0 if empty inputs occur.  Slower than lz_compress on inputs with
 * uneven chunks: a chunk whose offset is not yet known waits instead of
 * moving on. */
lz_status lz_compress_noalloc(const void *d_in, uint64_t n_bytes, const lz_params *p,
                              void *d_out, uint64_t out_cap, uint64_t *d_out_bytes,
                              lz_stream_t stream);

/* ---- Batches: many buffers in one persistent launch ------------------------
 * A batch is planned once on the host (lz_batch_create: validates every item,
 * uploads per-buffer descriptors, sizes and allocates its own scratch) and
 * run any number of times (lz_batch_run: a scratch clear and one persistent
 * kernel whose warps take chunks of all buffers from one work counter; no
 * host synchronisation, no allocation, so a run can be captured in a CUDA
 * graph and replayed).  The result of every item is byte-identical to
 * lz_compress / lz_decompress of that item alone.  Device errors are sticky
 * in the context, as for the single-buffer calls. */
typedef struct lz_batch_item {
  const void *d_in;      /* input (compress) or stream (decompress)         */
  uint64_t in_bytes;
  void *d_out;           /* output buffer                                   */
  uint64_t out_cap;
  uint64_t *d_out_bytes; /* device uint64, 8-byte aligned: produced size    */
  lz_params params;      /* compress: this item's parameters.  decompress:
                            all zero, or the stream's parameters (see
                            lz_batch_create)                                */
} lz_batch_item;

typedef struct lz_batch lz_batch;

/* Plan a batch of n_items over the host array `items` (decompress != 0: the
 * items are GLZ1 streams to decompress).  A decompression item whose
 * params.chunk_bytes is 0 has its header read from the device, which
 * synchronises `stream`; an item that states its stream's parameters in
 * `params` and its exact decompressed size in `out_cap` is planned without
 * that read (when every item does, the call does not synchronise), and the
 * kernel checks each header against the plan: a stream whose header
 * disagrees is not decoded and is reported as LZ_ERR_CORRUPT by lz_sync.
 * The batch's device memory is
 * allocated stream-ordered on `stream` (cudaMallocAsync) and its descriptors
 * uploaded on it, so no device-wide synchronisation happens; runs must be
 * ordered after this call (same stream, or an event).  Errors are those of
 * the single-buffer calls (checked per item) plus LZ_ERR_NOMEM, and
 * LZ_ERR_INVALID_ARG when a compression batch's items hold more than
 * 2^32 - 2^20 - 1 chunks together (one 32-bit work counter).  The buffers
 * named by the items must stay valid while the batch is run. */
lz_status lz_batch_create(lz_ctx *ctx, const lz_batch_item *items, uint32_t n_items,
                          int decompress, lz_stream_t stream, lz_batch **out);

/* lz_batch_create with options for a compression batch: every item is
 * compressed with opt->match and written as stream version opt->version,
 * exactly as lz_compress_ex with the same options would (opt NULL: the
 * defaults; ignored for a decompression batch, which reads both versions).
 * LZ_ERR_INVALID_ARG for the combinations lz_compress_ex rejects. */
lz_status lz_batch_create_ex(lz_ctx *ctx, const lz_batch_item *items, uint32_t n_items,
                             int decompress, const lz_options *opt, lz_stream_t stream,
                             lz_batch **out);

/* Re-plan a batch for new items of the same direction and options (those
 * given to lz_batch_create_ex), keeping its device memory where it is large
 * enough (a re-plan allocates only when the new items need more; every
 * buffer is allocated with room for half as much again).  The uploads are
 * ordered on `stream`, which must also order them after the batch's earlier
 * runs (the same stream, or an event).  Validation and errors as for
 * lz_batch_create; after a failed update the batch cannot be run until an
 * update succeeds.  A run captured in a CUDA graph before the update runs
 * the old plan's launch shape: capture again. */
lz_status lz_batch_update(lz_ctx *ctx, lz_batch *batch, const lz_batch_item *items,
                          uint32_t n_items, lz_stream_t stream);

/* Enqueue one run of the batch on `stream`. */
lz_status lz_batch_run(lz_ctx *ctx, lz_batch *batch, lz_stream_t stream);

/* Free a batch: its device memory is released stream-ordered on `stream`
 * (after the work already enqueued there); the handle is gone at once. */
void lz_batch_destroy(lz_batch *batch, lz_stream_t stream);

/* Choose chunk_bytes and window for data of `symbol_bytes`-byte symbols from
 * timed trial compressions of a device-resident sample: among C in {2048,
 * 4096, 8192, 16384} and W in {64, 128, 256, 512} whose compression ratio
 * is within 5% of the best ratio found, the smallest C that is within 10%
 * of the fastest time (less shared memory per warp, which helps a batched
 * launch over buffers of several kinds), then the fastest; min_match 3 (2
 * for 4-byte symbols), max_match 255.  The choice changes the stream (it is
 * recorded in its header), never the arithmetic: the stream is exactly
 * what lz_compress produces with the chosen parameters.  Synchronous;
 * allocates and frees temporary device buffers. */
lz_status lz_autotune(lz_ctx *ctx, const void *d_sample, uint64_t sample_bytes,
                      uint32_t symbol_bytes, lz_params *out);

/* One trial of lz_autotune_ex: the parameters, the launch shape
 * (lz_options.warps_per_block; 0 = the library's choice), the mean time of
 * one compression of the sample in seconds, and the compression ratio. */
typedef struct lz_tune_trial {
  lz_params params;
  uint32_t warps_per_block;
  double seconds;
  double ratio;
} lz_tune_trial;

/* lz_autotune, then the launch shape for the chosen parameters: warps per
 * block 1, 2, 4 and 8 (those that fit) are timed beside the library's own
 * choice, and the fastest is returned in *out_warps_per_block (0 when the
 * library's choice is within 2% of it); pass it in lz_options.  Every
 * trial (the 16 parameter sets, then the shapes) is written to trials[0 ..
 * min(max_trials, *n_trials)) and their count to *n_trials; either may be
 * NULL, as may out_warps_per_block. */
lz_status lz_autotune_ex(lz_ctx *ctx, const void *d_sample, uint64_t sample_bytes,
                         uint32_t symbol_bytes, lz_params *out, uint32_t *out_warps_per_block,
                         lz_tune_trial *trials, uint32_t max_trials, uint32_t *n_trials);

/* The paper's parameter selection (section 3.2.3), for data whose elements
 * are dtype_bytes wide (1, 2 or 4) at compression level `level` (1-4,
 * windows 32/64/128/255 symbols; a higher level gives a better ratio at a
 * lower throughput).  Multi-byte matching is the default: S = dtype_bytes
 * and the level's window enlarged S times (at most 1024).  The sample at
 * d_sample (device, sample_bytes rounded down to a multiple of
 * dtype_bytes) is compressed with it; when its compression ratio
 * (sample bytes / stream bytes) is below 1.5 the policy falls back to
 * single-byte matching, S = 1 with the level's window.  In both cases
 * C = chunk_bytes, M = 255 and m = the shortest profitable match,
 * (1 + offB) / S + 1 (integer division).  dtype_bytes = 1 needs no trial.
 * Writes the chosen parameters to *out.  Synchronises `stream`; allocates
 * and frees temporary device buffers (stream-ordered).  LZ_ERR_INVALID_ARG
 * for a bad dtype, level or chunk size or an empty sample. */
lz_status lz_select_params(lz_ctx *ctx, const void *d_sample, uint64_t sample_bytes,
                           uint32_t dtype_bytes, uint32_t level, uint32_t chunk_bytes,
                           lz_params *out, lz_stream_t stream);

/* Stitch one shard stream into a whole-input stream.  Chunks are
 * independent (section 3.3.1), so the stream of bytes [b0, b1) of an input
 * holds exactly the chunk records the whole-input stream holds for those
 * chunks when b0 is a multiple of 64 * chunk_bytes (one index superblock):
 * shards compressed separately (on several GPUs, or one after another) can
 * be placed side by side.  The one exchange between shards is the
 * exclusive scan of their (chunk count, record bytes); given it,
 *   d_shard, shard_bytes  the shard's GLZ1 stream (device, 8-byte aligned);
 *   shard_chunks          its chunk count (must equal its header's);
 *   chunk_base            chunks before it (a multiple of 64);
 *   total_chunks, total_bytes  the whole input's chunk and byte counts;
 *   record_base           record bytes of all earlier shards;
 *   d_out, out_cap        the whole-input stream (device, 8-byte aligned);
 * this call writes the shard's table entries, index entries (rebased by
 * record_base) and records at their places in d_out, and the header too
 * when chunk_base is 0.  Once every shard has been stitched, d_out holds
 * exactly the stream lz_compress writes for the whole input.  Argument and
 * range errors are returned synchronously; a shard header that disagrees
 * with the arguments (magic, version, chunk count, chunk count of
 * total_bytes) is LZ_ERR_CORRUPT from lz_sync and nothing is written.
 * The paper has no multi-GPU path: this is its chunk independence used
 * across shards. */
lz_status lz_stitch(lz_ctx *ctx, const void *d_shard, uint64_t shard_bytes,
                    uint64_t shard_chunks, uint64_t chunk_base, uint64_t total_chunks,
                    uint64_t total_bytes, uint64_t record_base, void *d_out,
                    uint64_t out_cap, lz_stream_t stream);

/* Synchronise `stream`, then return and clear the context's sticky device
 * error (LZ_OK if none).  When several errors occurred the most severe is
 * returned: INTERNAL, TIMEOUT, CORRUPT, then BUFFER_TOO_SMALL. */
lz_status lz_sync(lz_ctx *ctx, lz_stream_t stream);

/* ---- Test hooks --------------------------------------------------------------
 * For tests of the error paths only (no paper counterpart): they make a
 * bounded device wait run out, or an allocation fail, on purpose, without
 * faulting or hanging a GPU.  All zero (the state of a new context) means
 * normal operation; hooks == NULL resets them.  They apply to the context's
 * later calls:
 *   spin_limit  polls before a compression kernel's device waits give up
 *               (look-back and TMA staging; 0: the library's limit, about
 *               four million polls with back-off up to 1 us between
 *               look-back polls).  A wait that gives up raises
 *               LZ_ERR_TIMEOUT (returned by lz_sync) and the kernel
 *               finishes; the stream written is then incomplete.
 *   first_chunk lz_compress / lz_compress_ex hand out chunks from this one
 *               on, so chunks before it are never compressed and the
 *               look-back of the chunks after them waits for a prefix that
 *               never comes (with a small spin_limit: LZ_ERR_TIMEOUT).
 *   fail_alloc  when nonzero, every device allocation the context (or a
 *               batch planned on it) would make fails with LZ_ERR_NOMEM
 *               before anything is enqueued; memory already held is used.
 * LZ_ERR_INVALID_ARG for ctx == NULL. */
typedef struct lz_test_hooks {
  uint32_t spin_limit;
  uint32_t first_chunk;
  uint32_t fail_alloc;
} lz_test_hooks;

lz_status lz_set_test_hooks(lz_ctx *ctx, const lz_test_hooks *hooks);

/* ---- Huffman stage ----------------------------------------------------------
 * In the paper's use case (section 4.5) gpuLZ runs before cuSZ's Huffman
 * encoding.  The paper does not print that stage, so its definition here is
 * this library's: a byte-alphabet prefix code, optimal among codes whose
 * lengths do not exceed 12 bits (package-merge; ties: a leaf before a
 * package of equal weight, leaves by (count, value)), with canonical codes
 * (symbols in order of (length, value) take consecutive values).
 *
 * Stream "GHF1" (integers little-endian):
 *   [0,16)    "GHF1", u32 block bytes (32768), u64 n_bytes
 *   [16,272)  256 x u8: code length of each byte value (0 = absent)
 *   table     n_blocks x u64: end of each block's bit string, in bytes from
 *             the start of `bits`; block b spans [end[b-1], end[b])
 *   subs      n_blocks x 32 x u32: bit offset, inside its block, of each of
 *             its 32 sub-blocks of 1024 input bytes (sub-blocks past the end
 *             of the input repeat the end offset)
 *   bits      per block, a whole number of u32 words; bit i of a block is
 *             bit 31 - (i % 32) of its word i / 32; codes most significant
 *             bit first; padding bits 0.
 * n_blocks = ceil(n_bytes / 32768); `bits` starts at 272 + 136 n_blocks. */

/* Largest GHF1 stream for n_bytes of input (pure host). */
uint64_t lz_huff_bound(uint64_t n_bytes);

/* Huffman-code n_bytes at d_in (any alignment) into d_out (8-byte aligned,
 * capacity out_cap) and store the stream size in *d_out_bytes (device
 * uint64, 8-byte aligned).  Five launches (histogram, code book, sub-block
 * sizes, block offsets, encode); no host synchronisation.  out_cap below
 * the header and tables is LZ_ERR_BUFFER_TOO_SMALL at once; a stream that
 * does not fit is reported by lz_sync (LZ_ERR_BUFFER_TOO_SMALL) with the
 * size that was needed in *d_out_bytes.  lz_huff_bound(n_bytes) always
 * suffices.  Uses the context's scratch, like lz_compress. */
lz_status lz_huff_compress(lz_ctx *ctx, const void *d_in, uint64_t n_bytes, void *d_out,
                           uint64_t out_cap, uint64_t *d_out_bytes, lz_stream_t stream);

/* n_bytes of the GHF1 stream at d_in (reads its 16-byte header; synchronises
 * `stream`).  LZ_ERR_CORRUPT for a bad header or a stream shorter than its
 * tables. */
lz_status lz_huff_decompressed_size(const void *d_in, uint64_t in_bytes, uint64_t *h_n,
                                    lz_stream_t stream);

/* Decode the GHF1 stream at d_in (8-byte aligned, in_bytes long) into d_out
 * (capacity out_cap) and store n_bytes in *d_out_bytes.  One launch; the
 * kernel reads the header and tables itself.  A bad header, code lengths
 * that do not form a complete code, block ends or sub-block offsets that
 * disagree with the bits, or a code not in the table are LZ_ERR_CORRUPT;
 * out_cap < n_bytes is LZ_ERR_BUFFER_TOO_SMALL; both come from lz_sync. */
lz_status lz_huff_decompress(lz_ctx *ctx, const void *d_in, uint64_t in_bytes, void *d_out,
                             uint64_t out_cap, uint64_t *d_out_bytes, lz_stream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* GB300_LZ_H */
