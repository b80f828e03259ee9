/*
 * ORACLE -- test infrastructure only.
 *
 * A plain, slow, sequential CPU implementation of the two-layer codec of
 * "Unified Position-Invariant Random Access Through Two Compression Layers
 * via Absolute-Offset Coordinates" (ACEAPEX): an LZ77 match layer whose
 * back-references are absolute positions in the decompressed output
 * (Section 2, Section 3), output cut into fixed-size blocks (Section 2), the
 * separated token streams of each block entropy-coded with interleaved rANS
 * (Section 1, Section 3, Section 9), and the unified seek that decodes one
 * block through both layers from one absolute coordinate (Section 5).
 *
 * Only the test suite, the smoke check and the benchmark's CPU-baseline leg
 * may call this code.  It shares no source with the GPU library: its format
 * constants, table construction and arithmetic are written out here on their
 * own.
 *
 * Parity status of each part:
 *   rANS coder      pinned: round trip, state invariants, exact byte counts
 *                   for uniform tables, a hand-worked example
 *   LZ layer        pinned: brute-force round trip, longest-match check,
 *                   source-reproduces-destination check
 *   whole archive   pinned: decode equals the regenerated original
 *   stored streams  pinned: adaptive archives decode to the original, and a
 *                   stream is stored exactly when its rANS coding is no
 *                   smaller (checked against the rANS-only archive)
 *   seek            pinned: slice equals the original slice
 *   printed hashes  parity unpinned: the paper's FASTQ data (Section 5) is
 *                   not available, so its FNV values cannot be reproduced
 */
#ifndef ACE_ORACLE_H
#define ACE_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    ORC_OK = 0,
    ORC_E_INVAL = -1,
    ORC_E_CORRUPT = -2,
    ORC_E_RANGE = -3,
    ORC_E_NOMEM = -4,
};

uint64_t oracle_fnv1a64(const uint8_t *p, uint64_t n);
uint32_t oracle_fnv1a32(const uint8_t *p, uint64_t n);

/* rANS, one stream of n byte symbols over 32 interleaved 32-bit states */
int oracle_rans_freqs(const uint8_t *sym, uint32_t n, uint16_t freq[256]);
int oracle_rans_encode(const uint8_t *sym, uint32_t n, const uint16_t freq[256],
                       uint32_t states[32], uint8_t *out, uint32_t cap, uint32_t *out_len);
int oracle_rans_decode(const uint8_t *bytes, uint32_t nbytes, const uint32_t states[32],
                       const uint16_t freq[256], uint32_t n, uint8_t *sym);

/* whole archive */
uint64_t oracle_encode_bound(uint64_t n, uint32_t log2_block);
int oracle_encode(const uint8_t *in, uint64_t n, uint32_t log2_block, uint32_t min_match,
                  uint32_t max_chain, uint8_t *arc, uint64_t cap, uint64_t *arc_len);
int oracle_encode_adaptive(const uint8_t *in, uint64_t n, uint32_t log2_block, uint32_t min_match,
                           uint32_t max_chain, uint32_t adaptive, uint8_t *arc, uint64_t cap,
                           uint64_t *arc_len);
int oracle_info(const uint8_t *arc, uint64_t arc_len, uint64_t *total, uint32_t *block_size,
                uint64_t *n_blocks, uint32_t *off_width);
int oracle_decode(const uint8_t *arc, uint64_t arc_len, uint8_t *out, uint64_t out_cap);
int oracle_decode_block_tokens(const uint8_t *arc, uint64_t arc_len, uint64_t block,
                               uint32_t *lit_run, uint32_t *match_len, uint64_t *src,
                               uint32_t cap, uint32_t *ntok);
int oracle_levels(const uint8_t *arc, uint64_t arc_len, uint32_t *level);
int oracle_closure(const uint8_t *arc, uint64_t arc_len, uint64_t first, uint64_t last,
                   uint8_t *in_closure);
int oracle_seek(const uint8_t *arc, uint64_t arc_len, uint64_t coord, uint64_t len,
                uint8_t *out);

#ifdef __cplusplus
}
#endif
#endif
