/*
 * ace.h -- C ABI of the GPU library for the two-layer codec of "Unified
 * Position-Invariant Random Access Through Two Compression Layers via
 * Absolute-Offset Coordinates" (ACEAPEX).
 *
 * The codec stacks an LZ77 match layer whose back-references are absolute
 * positions in the decompressed output (Section 2, Section 3) under a
 * per-block interleaved-rANS entropy layer over separated literal, length
 * and offset streams (Section 3, Section 6.1, Section 9).  Because both
 * layers are entered at the block boundary, one absolute coordinate names
 * the entry point of both (Section 3), and a block decodes through both
 * layers once the blocks holding its match sources are present (Section 2).
 * The archive layout is in ace_format.h.
 *
 * Conventions for every call:
 *  - Pointers named d_* are device pointers, h_* host pointers.
 *  - The library never allocates device memory.  The caller sizes buffers
 *    with the *_size calls and owns them: the archive (which must outlive
 *    the index), the index memory, scratch and outputs.  The library owns
 *    only the small host handle that ace_index_free releases.
 *  - Device work is enqueued on the caller's stream and is asynchronous
 *    unless a call says otherwise.  Host-side validation errors return at
 *    once; errors found on the device (corrupt streams, a wait that gave up)
 *    are recorded in the scratch status word and returned by ace_sync.
 *  - Calls that share one scratch buffer must be ordered on one stream;
 *    calls with separate scratch buffers may overlap on the device.
 *  - The library keeps no global state except the CUDA device it runs on,
 *    taken as the current device when the index is built, and 256 KiB of
 *    pinned, mapped host memory allocated once per process on first use,
 *    through which the calls that report a device status read it back
 *    (a copy would queue behind other streams' large transfers).
 */
#ifndef ACE_H
#define ACE_H
#include <stddef.h>
#include <stdint.h>

#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t ace_status;
enum {
    ACE_OK = 0,
    ACE_E_INVAL = 1,   /* bad argument, null pointer, unaligned buffer */
    ACE_E_CORRUPT = 2, /* archive fails a structural or entropy check */
    ACE_E_RANGE = 3,   /* coordinate range outside the decompressed data */
    ACE_E_NOMEM = 4,   /* caller buffer or scratch too small */
    ACE_E_TIMEOUT = 5, /* a device-side wait gave up */
    ACE_E_CUDA = 6     /* a CUDA runtime call failed */
};

/* Name of a status code ("ACE_OK", ...); never NULL. */
const char *ace_status_str(ace_status s);

/* ------------------------------------------------------------ encoding */

typedef struct {
    uint32_t log2_block; /* block size 2^log2_block bytes, 8..16 (Section 2) */
    uint32_t min_match;  /* shortest match taken, >= 4 */
    uint32_t threads;    /* host threads; 0 = all hardware threads */
    uint32_t max_chain;  /* candidates tried per position in the in-block chain */
    uint32_t off_width;  /* absolute-offset bytes: 0 = 4 up to 2^32 input bytes, else 5; 5 forces 5; 4 above 2^32 is ACE_E_INVAL */
    uint32_t adaptive;   /* 1: store a block's stream verbatim (mode 1) when its rANS coding takes at least as many
                            bytes as its symbols (Section 6.1: entropy coding pays only on some streams); 0: rANS always */
} ace_encode_params;

/*
 * Host encoder (CPU).  Writes the archive of h_in[0, n) into h_arc:
 * greedy parse (Section 2's global match search: earliest occurrences of
 * 16-byte keys anywhere earlier in the input, plus shorter repeats inside
 * the block), stream separation, per-block rANS with 32 interleaved 32-bit
 * states, 12-bit frequencies and byte renormalisation (Section 3), and the
 * block dependency table.  ace_encode_bound gives a size that always
 * suffices.  Returns ACE_E_INVAL for bad parameters, ACE_E_NOMEM when cap is
 * too small.  Deterministic: the archive does not depend on the thread count.
 */
ace_status ace_encode_bound(uint64_t n, uint32_t log2_block, uint64_t *bound);
ace_status ace_encode(const void *h_in, uint64_t n, const ace_encode_params *params,
                      void *h_arc, uint64_t cap, uint64_t *arc_len);

/*
 * The same encoder in two steps, for inputs whose bound is too large to
 * allocate: ace_encode_run encodes into library-owned host memory and
 * reports the exact archive size; ace_encode_write copies the archive out
 * (cap >= that size); ace_encode_free releases the encoder.
 */
typedef struct ace_encoder ace_encoder;
ace_status ace_encode_run(const void *h_in, uint64_t n, const ace_encode_params *params,
                          ace_encoder **out, uint64_t *arc_len);
ace_status ace_encode_write(const ace_encoder *enc, void *h_arc, uint64_t cap);
ace_status ace_encode_free(ace_encoder *enc);

/* What the parse produced, for reporting: tokens, matches, literal and match
 * bytes, match_src_bytes = sum over matches of min(length, distance) (the
 * distinct source bytes a decoder must read), dependency intervals and
 * levels (1 + the deepest block level). */
typedef struct {
    uint64_t n_tokens;
    uint64_t n_matches;
    uint64_t literal_bytes;
    uint64_t match_bytes;
    uint64_t match_src_bytes;
    uint64_t n_dep_intervals;
    uint32_t n_levels;
    uint32_t reserved;
} ace_encode_stats;
ace_status ace_encode_get_stats(const ace_encoder *enc, ace_encode_stats *h_stats);

/*
 * GPU encoder: the whole encode on the device, from d_in[0, n) (device
 * memory) to an archive in d_arc (device memory, 256-byte aligned) in the
 * layout of ace_format.h.  Section 2's global match search as a table of
 * the earliest occurrence of every 16-byte key at 8-byte strides (built with
 * atomic minima), in-block repeats through 4-byte hash chains (a warp per
 * block), candidates measured for every position at once (a thread per
 * position), then a greedy walk per block (a thread per block) that takes
 * the longest allowed candidate, refusing in-block resolution waves deeper
 * than 3 and preferring a shallower candidate nearly as long; blocks in
 * windows of 64 that take no sources from each other, the first three
 * windows in order, every later block taking external sources only from
 * them (dependency levels at most 3).  Each block's literal, length and
 * offset streams rANS-coded by a warp (Section 3; the host encoder's
 * frequency quantisation, 32 interleaved states), stored verbatim with
 * params->adaptive where rANS would not shrink them (Section 6.1).  The
 * parse differs from the host encoder's; every decoder reads both.
 * params->threads is read as the blocks parsed per launch (0: 64 MiB of
 * input's worth); max_chain <= 64.  ace_encode_gpu_size gives the scratch
 * (256-byte aligned) and a d_arc size that always suffices; a smaller d_arc
 * may do (the archive plus room for the largest dependency table), and the
 * call returns ACE_E_NOMEM when it does not.  Synchronises s; *h_arc_len
 * gets the archive's bytes, h_stats (may be NULL) the parse statistics.
 */
ace_status ace_encode_gpu_size(uint64_t n, const ace_encode_params *params, uint64_t *scratch_bytes,
                               uint64_t *arc_bound);
ace_status ace_encode_gpu(const void *d_in, uint64_t n, const ace_encode_params *params, void *d_scratch,
                          uint64_t scratch_bytes, void *d_arc, uint64_t arc_cap, uint64_t *h_arc_len,
                          ace_encode_stats *h_stats, cudaStream_t s);

/* ------------------------------------------------------------ the index */

typedef struct ace_index ace_index;

typedef struct {
    uint64_t total_size;    /* decompressed bytes */
    uint64_t n_blocks;
    uint64_t archive_bytes;
    uint64_t n_dep_intervals;
    uint32_t block_size;
    uint32_t off_width;
    uint32_t n_levels;      /* dependency levels: 1 + the deepest level */
    uint32_t reserved;
} ace_info;

/*
 * Bytes of device memory the index of an archive needs, from its 64-byte
 * header (h_header, header_bytes >= 64).  ACE_E_CORRUPT for a header that
 * is not a version-1 archive.
 */
ace_status ace_index_size(const void *h_header, uint64_t header_bytes, uint64_t *index_bytes);

/*
 * Builds the block index on the device (Section 3: the block boundary is
 * the entry point of both layers; Section 2: a block decodes once the blocks
 * holding its sources are present): validates every directory entry and the
 * dependency table, computes each block's dependency level (0 without
 * sources in other blocks, else 1 + the deepest source block) and the decode
 * order (level, then block).  d_archive holds archive_bytes bytes (16-byte
 * aligned), h_header its first 64 bytes on the host.  d_index_mem (256-byte
 * aligned, index_bytes from ace_index_size) is written by this call and
 * only read afterwards.  Synchronises s before it returns; on success *out is
 * a new handle.  ACE_E_CORRUPT when the archive fails validation.
 */
ace_status ace_index_build(const void *d_archive, uint64_t archive_bytes, const void *h_header,
                           uint64_t header_bytes, void *d_index_mem, uint64_t index_bytes,
                           cudaStream_t s, ace_index **out);

/* Fills h_info from the host handle (no device access). */
ace_status ace_index_info(const ace_index *idx, ace_info *h_info);

/* Blocks per dependency level (Section 2's decode order), for the first
 * min(n, n_levels) levels, into h_counts.  Synchronises s when the counts
 * live only on the device (archives with more than 32 levels). */
ace_status ace_index_levels(const ace_index *idx, uint32_t *h_counts, uint32_t n, cudaStream_t s);

/* Releases the host handle; the caller frees the device buffers. */
ace_status ace_index_free(ace_index *idx);

/*
 * A stored index: the index memory written to host bytes (h_blob, for a
 * file) so that a later process loads it instead of rebuilding it (the
 * storage format of Section 8's next step: a prepared archive and its index
 * loaded from disk).  ace_index_export_size gives the bytes;
 * ace_index_export copies the index memory after a 256-byte header holding
 * the archive's header and an FNV-1a 64 of the index bytes, and
 * synchronises s.  ace_index_import takes the same arguments as
 * ace_index_build plus the blob: it checks that the blob belongs to this
 * archive and is whole (ACE_E_CORRUPT otherwise), copies it to d_index_mem,
 * and, instead of iterating the level rule, verifies the stored levels
 * against the archive's dependency table in one sweep and the stored order
 * as a level-sorted permutation of the blocks; the archive's directory is
 * validated as at a build.  Synchronises s; on success *out is a new handle.
 */
ace_status ace_index_export_size(const ace_index *idx, uint64_t *bytes);
ace_status ace_index_export(const ace_index *idx, void *h_blob, uint64_t blob_bytes, cudaStream_t s);
ace_status ace_index_import(const void *d_archive, uint64_t archive_bytes, const void *h_header, uint64_t header_bytes,
                            const void *h_blob, uint64_t blob_bytes, void *d_index_mem, uint64_t index_bytes,
                            cudaStream_t s, ace_index **out);

/*
 * Archives larger than device memory (Section 7: the output and the archive
 * together exceed VRAM, so ranges are decoded instead).  The archive may
 * stay in host memory: ace_host_register pins and maps h_p[0, bytes) (a file
 * read or mapped into memory) and returns in *d_p the address the GPU reads
 * it through (over the chip-to-chip link on Grace hosts); pass *d_p as
 * d_archive to ace_index_build or ace_index_import, and seek ranges of it as
 * usual.  read_only = 1 for archives (the GPU never writes them); 0 for a
 * host buffer that decodes write into.  ace_host_unregister undoes it, after
 * every call that reads the memory has finished.  This pins host memory; it
 * allocates no device memory.  ACE_E_CUDA when the runtime refuses.
 */
ace_status ace_host_register(void *h_p, uint64_t bytes, uint32_t read_only, void **d_p);
ace_status ace_host_unregister(void *h_p);

/* ------------------------------------------------------------- scratch */

/*
 * Scratch bytes for one call on this index.  max_seek_blocks is the largest
 * number of blocks a seek may decode (its target blocks plus every block
 * they read from, transitively); 0 sizes scratch for ace_decode_all only.
 * Scratch must be 256-byte aligned.  Its first use must follow
 * ace_scratch_init on the same stream.
 */
ace_status ace_scratch_size(const ace_index *idx, uint64_t max_seek_blocks, uint64_t *bytes);

/* Clears scratch (asynchronous on s). */
ace_status ace_scratch_init(const ace_index *idx, void *d_scratch, uint64_t scratch_bytes,
                            cudaStream_t s);

/* ------------------------------------------------------------ decoding */

/* How a decode is laid out in launches.
 * ACE_SCHEDULE_PASSES: three passes -- tokens (length and offset streams
 * into match records) and literals as persistent launches over the blocks,
 * then the match pass, one launch per dependency level.
 * ACE_SCHEDULE_FUSED: one persistent launch.  Each warp takes a block in
 * (level, block) order and decodes its entropy layer, then holds the
 * block's matches until every block of the lower levels is resolved,
 * taking further blocks meanwhile (at most four held), so the entropy
 * decode of some warps overlaps the match copies of others.
 * ACE_SCHEDULE_AUTO (0): the library's choice, currently the passes.
 * Seek batches through a block cache always run the passes; plain seeks
 * take the fused schedule only for archives of at most 32 levels. */
enum { ACE_SCHEDULE_AUTO = 0, ACE_SCHEDULE_PASSES = 1, ACE_SCHEDULE_FUSED = 2 };

typedef struct {
    uint32_t warps_per_cta;   /* 1..8; 0 = default (4) */
    uint32_t ctas_per_sm;     /* 0 = as many as fit */
    uint32_t chunk_tokens;    /* tokens staged per step, 32..256, multiple of 32; 0 = 128 */
    uint32_t schedule;        /* ACE_SCHEDULE_*; 0 = automatic; others: ACE_E_INVAL */
    uint64_t wait_timeout_ns; /* bound on each device-side wait; 0 = 2 s */
    uint32_t copy_width;      /* match copies: 16 = every non-overlapping match above 32 bytes in aligned
                                 16-byte pieces; 8 = 8-byte words up to 32 bytes, bytewise up to 511,
                                 16-byte pieces from 512; 0 = the library's choice (16); others: ACE_E_INVAL */
    uint32_t reserved;        /* 0 */
} ace_tune;

/*
 * Whole-archive decode through both layers (Sections 2-3) into d_out
 * (16-byte aligned, out_bytes >= total_size), on s.  Each block's length and offset streams
 * are rANS-decoded into one record per match (absolute source, destination,
 * length), its literal stream is decoded straight to its positions in
 * d_out, and its absolute-offset matches are resolved once the blocks they
 * read are present (Section 2).  The pass schedule (the default) runs three
 * passes: tokens and literals as persistent launches over the blocks, then
 * the match pass one launch per dependency level (a CTA per block for levels
 * of at most two blocks per SM and blocks of at most 32 KiB, a warp per
 * block otherwise), or, for archives of more than 32 levels, one persistent
 * launch in (level, block) order with bounded waits on source blocks' ready
 * flags.  ACE_SCHEDULE_FUSED does all of it in one persistent launch.
 * A source block whose level is not below its reader's makes the call
 * report ACE_E_CORRUPT.  tune may be NULL.  Asynchronous; check with
 * ace_sync.
 */
ace_status ace_decode_all(const ace_index *idx, void *d_out, uint64_t out_bytes, void *d_scratch,
                          uint64_t scratch_bytes, const ace_tune *tune, cudaStream_t s);

/*
 * The passes of ace_decode_all's pass schedule as separate calls, so that a
 * caller can time each one with events on s: ACE_PASS_TOKENS (which also
 * resets the call's status), ACE_PASS_LITERALS, then ACE_PASS_MATCH, same
 * arguments, same stream; together they are exactly ace_decode_all with
 * ACE_SCHEDULE_PASSES.  Any other pass value: ACE_E_INVAL.
 */
enum { ACE_PASS_TOKENS = 0, ACE_PASS_LITERALS = 1, ACE_PASS_MATCH = 2 };
ace_status ace_decode_pass(const ace_index *idx, int pass, void *d_out, uint64_t out_bytes, void *d_scratch,
                           uint64_t scratch_bytes, const ace_tune *tune, cudaStream_t s);

/*
 * Unified seek (Section 5): the absolute range [coord, coord + len) names
 * its covering blocks; they and every block their matches read,
 * transitively, are decoded from the archive alone into scratch, and exactly
 * the len requested bytes are written to d_out[0, len).  Nothing else in
 * d_out is touched.  coord and len need no alignment.  ACE_E_RANGE when
 * len == 0 or coord + len > total_size.  If the blocks to decode exceed the
 * max_seek_blocks the scratch was sized for, ace_sync reports ACE_E_NOMEM;
 * if a match reads a block outside that set (the archive's dependency lists
 * disagree with its matches), ace_sync reports ACE_E_CORRUPT.  Asynchronous.
 */
ace_status ace_seek(const ace_index *idx, uint64_t coord, uint64_t len, void *d_out,
                    uint64_t out_bytes, void *d_scratch, uint64_t scratch_bytes, cudaStream_t s);

/* Sets the tuning ace_seek uses, and ace_decode_all when given no tune
 * (NULL restores the defaults).  Not thread-safe against calls in flight on
 * the host. */
ace_status ace_index_set_tune(ace_index *idx, const ace_tune *tune);

/* Synchronises s and returns (then clears) the first device-side error
 * recorded in the scratch status word. */
ace_status ace_sync(const ace_index *idx, void *d_scratch, cudaStream_t s);

/* ---------------------------------------------------------------- batches */

/*
 * Many independent archives decoded in one persistent launch (the batching
 * pattern: thousands of uneven objects with mixed block sizes).  Each
 * archive's blocks keep their own (level, block) order; warps take
 * (archive, block) items from one ticket, so a warp only waits on blocks of
 * its own archive handed out before it (Section 2's dependency rule).
 *
 * ace_batch_scratch_size sizes the batch scratch (256-byte aligned).
 * ace_batch_create records the archives (all on the current device) and
 * their outputs (16-byte aligned, out_bytes[i] >= the archive's total size;
 * ACE_E_INVAL for an unaligned one) in the scratch,
 * plans the launch from tune (NULL = defaults), and synchronises s.  It
 * allocates no device memory.  ace_decode_batch then enqueues, with no host
 * synchronisation, a header reset and the token, literal and match passes
 * (pass schedule) or a memset of the level counters, a header reset and one
 * fused launch (ACE_SCHEDULE_FUSED), so it can be captured into a CUDA graph
 * and replayed; each replay decodes every archive again.
 * ace_batch_sync synchronises s and returns (then clears) the first device
 * error.  ace_batch_launch_shape reports the planned grid, warps per CTA and
 * token window.
 */
typedef struct ace_batch ace_batch;
ace_status ace_batch_scratch_size(const ace_index *const *idx, uint32_t n, uint64_t *bytes);
ace_status ace_batch_create(const ace_index *const *idx, uint32_t n, void *const *d_outs,
                            const uint64_t *out_bytes, void *d_scratch, uint64_t scratch_bytes,
                            const ace_tune *tune, cudaStream_t s, ace_batch **out);
ace_status ace_decode_batch(const ace_batch *batch, cudaStream_t s);
ace_status ace_batch_sync(const ace_batch *batch, cudaStream_t s);
ace_status ace_batch_launch_shape(const ace_batch *batch, uint32_t *grid, uint32_t *warps_per_cta,
                                  uint32_t *window);
ace_status ace_batch_free(ace_batch *batch);

/* --------------------------------------------- seek batches and the cache */

/*
 * Many seeks, over several resident archives, in one pass: the serving
 * pattern.  A decoded-block cache (caller memory) holds n_slots decoded
 * blocks; every archive attached to it has a small per-archive state (ready
 * flags, slot map, closure marks, work positions; ace_archive_state_size).
 * A seek batch:
 *   1. finds every target block that is not cached and, transitively, every
 *      uncached block their matches read (Section 2), in ascending block
 *      order per archive, and gives each a slot from a clock over the slots:
 *      slots the batch itself uses are passed over, a slot used since the
 *      hand last passed it gets a second chance, and a slot taken from a
 *      cached block evicts that block;
 *   2. decodes those blocks through both layers into their slots (Section 3
 *      entry point, Section 2 match layer), waiting bounded on sources;
 *   3. copies each request's bytes [coord, coord + len) to d_pool + out_off.
 * Blocks stay cached across batches until evicted.  A batch whose new
 * blocks exceed the blocks one batch may decode (ace_cache_limits) or the
 * slots it does not use itself records ACE_E_NOMEM and copies nothing; the
 * cache stays valid, and the caller submits fewer requests (a single
 * request that still fails can never be served by this cache).  After any
 * other error, call ace_cache_reset (every block uncached, every slot free).
 *
 * All archives of a cache share one device and one block size.  Batches on
 * one cache must be ordered on one stream; separate caches (each with its
 * own per-archive states) may run concurrently on separate streams.
 * ace_seek_batch reads device-resident requests and enqueues three kernels
 * plus the passes; ace_seek_batch_host validates host requests against the
 * archives' sizes (h_totals, may be NULL) and the pool, stages them in the
 * cache memory (n <= max_reqs) and calls it.  ace_cache_sync returns (then
 * clears) the first device error; ace_cache_usage reports slots holding a
 * block; ace_cache_counters the blocks evicted and decoded since creation;
 * ace_cache_limits the slots, the blocks one batch may decode and the
 * requests one batch may hold.
 */
typedef struct {
    uint32_t archive;  /* position of the archive in the cache's list */
    uint32_t reserved;
    uint64_t coord;    /* first absolute byte */
    uint64_t len;      /* bytes, >= 1 */
    uint64_t out_off;  /* byte offset of the result in the output pool */
} ace_seek_req;

typedef struct ace_cache ace_cache;
ace_status ace_archive_state_size(const ace_index *idx, uint64_t *bytes);
ace_status ace_cache_size(const ace_index *const *idx, uint32_t n, uint64_t n_slots, uint32_t max_reqs,
                          uint64_t *bytes);
ace_status ace_cache_create(const ace_index *const *idx, uint32_t n, void *const *d_states,
                            uint64_t n_slots, uint32_t max_reqs, void *d_mem, uint64_t bytes,
                            const ace_tune *tune, cudaStream_t s, ace_cache **out);
ace_status ace_seek_batch(const ace_cache *cache, const ace_seek_req *d_reqs, uint32_t n, void *d_pool,
                          uint64_t pool_bytes, cudaStream_t s);
ace_status ace_seek_batch_host(const ace_cache *cache, const ace_seek_req *h_reqs, const uint64_t *h_totals,
                               uint32_t n, void *d_pool, uint64_t pool_bytes, cudaStream_t s);
ace_status ace_cache_sync(const ace_cache *cache, cudaStream_t s);
ace_status ace_cache_usage(const ace_cache *cache, uint32_t *used_slots, uint32_t *n_slots, cudaStream_t s);
ace_status ace_cache_reset(const ace_cache *cache, cudaStream_t s);
ace_status ace_cache_counters(const ace_cache *cache, uint64_t *h_evicted, uint64_t *h_decoded, cudaStream_t s);
ace_status ace_cache_limits(const ace_cache *cache, uint32_t *h_n_slots, uint32_t *h_max_work, uint32_t *h_max_reqs);
ace_status ace_cache_free(ace_cache *cache);

/* ---------------------------------------------------------- verification */

typedef struct {
    uint64_t fnv_before;     /* FNV-1a 64 of the poisoned slice before the seek */
    uint64_t fnv_after;      /* FNV-1a 64 of the slice after the seek */
    uint64_t guard_bad_before; /* guard bytes differing from the canary, before */
    uint64_t guard_bad_after;  /* ... and after the seek */
    int32_t phase1_ok;       /* fnv_before != expected: the slice held no original data */
    int32_t phase2_ok;       /* fnv_after == expected: the seek produced the original */
    int32_t phase3_ok;       /* no guard byte changed: neighbours untouched */
    ace_status seek_status;  /* ace_sync result of the seek */
} ace_verify_report;

/*
 * The three-phase check of Section 5.  d_buf holds guard_bytes, then len
 * bytes for the slice, then guard_bytes.  The guards are filled with a
 * canary pattern from canary_seed and the slice with a different poison
 * pattern; phase 1 checks the slice's FNV-1a 64 differs from
 * expected_fnv1a64, the seek runs, phase 2 checks the slice's FNV equals it,
 * phase 3 checks every guard byte still holds its canary.  Synchronous.
 */
ace_status ace_verify(const ace_index *idx, uint64_t coord, uint64_t len, void *d_buf,
                      uint64_t guard_bytes, uint64_t expected_fnv1a64, uint32_t canary_seed,
                      void *d_scratch, uint64_t scratch_bytes, ace_verify_report *h_rep,
                      cudaStream_t s);

/* FNV-1a 64 (Fowler/Noll/Vo; the paper's bit-perfect check, Section 4) of
 * d_p[0, n), computed on the device into *d_result (8 bytes, device memory).
 * Asynchronous. */
ace_status ace_fnv1a64(const void *d_p, uint64_t n, uint64_t *d_result, cudaStream_t s);

/* ----------------------------------------------- seek without allocation */

/*
 * ace_seek without any device memory from the caller beyond the output:
 * for callers that cannot allocate device memory at all (a host application
 * that owns all device memory through its own pool, a plug-in inside such
 * an application, a request thread that must never reach the allocator).
 * The paper has no counterpart; it is a deployment convenience.
 *
 * Scratch comes from a fixed 32 MiB array in the library's device image,
 * held on every GPU that loads the library until the process exits, and
 * shared by every call on that device: calls that overlap on the GPU race,
 * so order them (one stream, or events).  The first call on a device looks
 * up the array's device address; make that first call before any stream
 * capture.  The index's device must be current.  Archives whose per-block
 * tables do not fit, or requests covering more blocks than the remaining
 * slots, return ACE_E_NOMEM.  Calls no allocator (the
 * status buffer above already exists once an index was built).
 * Synchronises s and returns the seek's device-side status (ACE_OK,
 * ACE_E_CORRUPT, ACE_E_TIMEOUT, ACE_E_NOMEM when the closure exceeds the
 * slots); otherwise as ace_seek.
 */
ace_status ace_seek_noalloc(const ace_index *idx, uint64_t coord, uint64_t len, void *d_out,
                            uint64_t out_bytes, cudaStream_t s);

#ifdef __cplusplus
}
#endif
#endif
