/*
 * ace_format.h -- byte layout of an archive of the two-layer codec, as read by
 * the GPU library and written by its host encoder.
 *
 * The paper fixes the structure (Section 2: absolute-offset LZ77 over fixed
 * blocks with separated token streams; Section 3: each block's streams
 * entropy-coded on their own, so the block boundary is the entry point of
 * both layers) but prints no byte format; this is the layout adopted.  All
 * integers are little-endian.
 *
 *   [0, 64)                   ace_file_header
 *   [dir_off, +64 n_blocks)   ace_block_dir, one per block
 *   [deps_off, ...)           u32 dep_ptr[n_blocks + 1], then u32 pairs
 *                             (first, last): for block b, entries
 *                             [dep_ptr[b], dep_ptr[b+1]) are the maximal runs
 *                             of earlier blocks its matches read
 *   [payload_off, ...)        stream payloads, each 16-byte aligned
 *   archive_bytes             total length, a multiple of 16
 *
 * Stream payload (mode 0, nsym > 0):
 *   u32 states[32]            final encoder state of each interleaved lane:
 *                             the decoder's entry point for this block
 *   u8  present[32]           bit s%8 of byte s/8 set when symbol s occurs
 *   u16 freq[k]               frequency of each present symbol, ascending
 *                             symbol order, sum 4096; zero-padded to a
 *                             multiple of 8 entries (16 bytes)
 *   u8  renorm[]              renormalisation bytes in decode order
 * Stream payload (mode 1, stored): the nsym symbols verbatim,
 *   stream_bytes = nsym, 16-byte aligned like every stream; for streams that
 *   rANS would not shrink (entropy coding chosen per stream at encode time,
 *   Section 6.1).
 * A stream with nsym = 0 has stream_bytes = 0 and no payload.
 *
 * Token streams of one block:
 *   0 literals   the literal bytes in output order
 *   1 lengths    nesc u16 escape values, then 2 codes per token
 *                (lit_run, match_len); code < 255 is the value, code 255
 *                takes the next escape value e and means 255 + e
 *   2 offsets    for every token but the last: the match's absolute source
 *                position in the decompressed output, off_width bytes
 * The last token of a block has match_len 0.  A match's destination lies in
 * its own block; its source precedes its destination and may overlap it
 * (sequential LZ77 semantics).
 */
#ifndef ACE_FORMAT_H
#define ACE_FORMAT_H
#include <stdint.h>

#define ACE_MAGIC 0x41454341u /* "ACEA" */
#define ACE_VERSION 1
#define ACE_NSTREAMS 3
#define ACE_NSTATES 32
#define ACE_SCALE_BITS 12
#define ACE_SCALE (1u << ACE_SCALE_BITS)
#define ACE_RANS_L (1u << 23)
#define ACE_MIN_LOG2_BLOCK 8
#define ACE_MAX_LOG2_BLOCK 16
#define ACE_STREAM_HEAD 160u /* states + present bitmap */

enum { ACE_S_LIT = 0, ACE_S_LEN = 1, ACE_S_OFF = 2 };

typedef struct {
    uint32_t magic;
    uint16_t version;
    uint8_t n_streams;
    uint8_t n_states;
    uint8_t scale_bits;
    uint8_t off_width;
    uint8_t log2_block;
    uint8_t reserved0;
    uint32_t flags;
    uint64_t total_size;
    uint64_t n_blocks;
    uint64_t dir_off;
    uint64_t deps_off;
    uint64_t payload_off;
    uint64_t archive_bytes;
} ace_file_header; /* 64 bytes */

typedef struct {
    uint64_t stream_off[3];   /* relative to payload_off */
    uint32_t stream_bytes[3];
    uint32_t nsym[3];
    uint32_t ntok;
    uint32_t nesc;
    uint8_t mode[3];          /* 0 = rANS, 1 = stored; others rejected */
    uint8_t reserved[5];
} ace_block_dir; /* 64 bytes */

#ifdef __cplusplus
static_assert(sizeof(ace_file_header) == 64, "header layout");
static_assert(sizeof(ace_block_dir) == 64, "directory layout");
#endif

#endif
