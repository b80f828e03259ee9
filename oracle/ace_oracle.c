/*
 * ORACLE -- test infrastructure only.  See ace_oracle.h for what it covers
 * and how each part is pinned.  Everything here is deliberately plain:
 * sequential loops, linear scans, bytewise copies, no blocking or fusion.
 *
 * Archive layout (the reading adopted where the paper gives no format; all
 * integers little-endian):
 *   header, 64 bytes: "ACEA", u16 version=1, u8 n_streams=3, u8 n_states=32,
 *     u8 scale_bits=12, u8 off_width (4, or 5 above 2^32 bytes),
 *     u8 log2_block, u8 0, u32 flags=0, u64 total_size, u64 n_blocks,
 *     u64 dir_off, u64 deps_off, u64 payload_off, u64 archive_bytes
 *   directory, 64 bytes per block: u64 stream_off[3] (relative to
 *     payload_off), u32 stream_bytes[3], u32 nsym[3], u32 ntok, u32 nesc,
 *     u8 mode[3], 5 zero bytes.  Stream 0 = literals, 1 = lengths,
 *     2 = absolute offsets.  mode 0: rANS-coded; mode 1: stored, the
 *     stream's symbols verbatim (stream_bytes = nsym), for streams that
 *     rANS would not shrink (Section 4: entropy coding applied per stream,
 *     measured at encode time).
 *   dependencies: u32 dep_ptr[n_blocks+1], then u32 (first, last) block
 *     pairs: the maximal runs of earlier blocks each block's matches read.
 *   payload: per non-empty stream, 16-byte aligned: u32 states[32],
 *     32-byte present-symbol bitmap, u16 freq per present symbol (ascending
 *     symbol order, zero-padded to a multiple of 16 bytes), renorm bytes
 *     (mode 0), or the symbols themselves (mode 1).
 * Token streams of a block:
 *   literals: the literal bytes in output order;
 *   lengths:  first nesc u16 escape values, then two one-byte codes per token
 *     (lit_run, match_len); a code < 255 is the value, code 255 takes the next
 *     escape value e and means 255 + e;
 *   offsets:  for every token but the last, the absolute source position of
 *     its match as off_width bytes.
 *   The last token of a block has match_len 0; a match never writes past the
 *   end of its block (Section 2: fixed-size blocks, absolute offsets).
 */
#include "ace_oracle.h"

#include <stdlib.h>
#include <string.h>

#define ORC_SCALE_BITS 12
#define ORC_M (1u << ORC_SCALE_BITS) /* frequency total, 4096 */
#define ORC_L (1u << 23)             /* lower bound of a normalised state */
#define ORC_LANES 32
#define ORC_HDR 64
#define ORC_DIR 64
#define ORC_NSTREAM 3
enum { S_LIT = 0, S_LEN = 1, S_OFF = 2 };

/* ----------------------------------------------------- little-endian io */

static uint64_t rd(const uint8_t *p, int nbytes)
{
    uint64_t v = 0;
    for (int i = nbytes - 1; i >= 0; i--) v = (v << 8) | p[i];
    return v;
}

static void wr(uint8_t *p, uint64_t v, int nbytes)
{
    for (int i = 0; i < nbytes; i++) { p[i] = (uint8_t)(v & 0xff); v >>= 8; }
}

static uint64_t align16(uint64_t v) { return (v + 15) & ~(uint64_t)15; }

/* ------------------------------------------------------------------ FNV */

/*
 * FNV-1a (Fowler, Noll, Vo): for each byte, xor it into the hash, then
 * multiply by the FNV prime.  The paper checks decoded output bit-perfect by
 * FNV hash (Section 4, Section 5); its 16-hex-digit value is FNV-1a 64.
 */
uint64_t oracle_fnv1a64(const uint8_t *p, uint64_t n)
{
    uint64_t h = 0xcbf29ce484222325ULL;
    for (uint64_t i = 0; i < n; i++) { h ^= p[i]; h *= 0x100000001b3ULL; }
    return h;
}

uint32_t oracle_fnv1a32(const uint8_t *p, uint64_t n)
{
    uint32_t h = 0x811c9dc5u;
    for (uint64_t i = 0; i < n; i++) { h ^= p[i]; h *= 0x01000193u; }
    return h;
}

/* ----------------------------------------------------------------- rANS */

/*
 * Quantised frequencies for one stream (the per-block entropy layer,
 * Section 3).  f_s = max(1, floor(n_s * 4096 / n)) for each present symbol;
 * a shortfall is added to the most frequent symbol (lowest value on ties);
 * an excess is removed one at a time from the symbol with the largest
 * frequency above 1 (lowest value on ties).  Sum is exactly 4096.
 */
int oracle_rans_freqs(const uint8_t *sym, uint32_t n, uint16_t freq[256])
{
    uint64_t cnt[256] = {0};
    for (uint32_t i = 0; i < n; i++) cnt[sym[i]]++;
    memset(freq, 0, 256 * sizeof(uint16_t));
    if (n == 0) return ORC_OK;
    int64_t sum = 0;
    int most = -1;
    for (int s = 0; s < 256; s++) {
        if (!cnt[s]) continue;
        uint64_t f = cnt[s] * ORC_M / n;
        if (f < 1) f = 1;
        freq[s] = (uint16_t)f;
        sum += (int64_t)f;
        if (most < 0 || cnt[s] > cnt[most]) most = s;
    }
    if (sum < (int64_t)ORC_M) freq[most] = (uint16_t)(freq[most] + (ORC_M - sum));
    while (sum > (int64_t)ORC_M) {
        int big = -1;
        for (int s = 0; s < 256; s++)
            if (freq[s] > 1 && (big < 0 || freq[s] > freq[big])) big = s;
        freq[big]--;
        sum--;
    }
    return ORC_OK;
}

static void cumulative(const uint16_t freq[256], uint32_t cum[257])
{
    cum[0] = 0;
    for (int s = 0; s < 256; s++) cum[s + 1] = cum[s] + freq[s];
}

/*
 * Interleaved rANS encoder (interleaved rANS, Section 1 and Section 9; per
 * block entry from the block boundary, Section 3).  Symbol i belongs to
 * state (lane) i mod 32.  All states start at L = 2^23.  Symbols are
 * encoded from the last to the first; before encoding symbol s with
 * frequency f, the state emits its low byte while x >= 2^19 * f, then
 * x <- floor(x / f) * 4096 + (x mod f) + c_s.  The emitted bytes are
 * reversed, so the decoder reads them forward in symbol order.  The final
 * states are stored; they are the decoder's entry point.
 */
int oracle_rans_encode(const uint8_t *sym, uint32_t n, const uint16_t freq[256],
                       uint32_t states[32], uint8_t *out, uint32_t cap, uint32_t *out_len)
{
    uint32_t cum[257];
    cumulative(freq, cum);
    if (n > 0 && cum[256] != ORC_M) return ORC_E_INVAL;
    uint64_t x[ORC_LANES];
    for (int j = 0; j < ORC_LANES; j++) x[j] = ORC_L;
    uint32_t len = 0;
    for (uint32_t k = n; k-- > 0;) {
        uint32_t s = sym[k], f = freq[s];
        if (f == 0) return ORC_E_INVAL;
        uint64_t *xs = &x[k % ORC_LANES];
        uint64_t xmax = ((uint64_t)(ORC_L >> ORC_SCALE_BITS) << 8) * f;
        while (*xs >= xmax) {
            if (len >= cap) return ORC_E_NOMEM;
            out[len++] = (uint8_t)(*xs & 0xff);
            *xs >>= 8;
        }
        *xs = (*xs / f) * ORC_M + (*xs % f) + cum[s];
    }
    for (uint32_t i = 0; i < len / 2; i++) {
        uint8_t t = out[i];
        out[i] = out[len - 1 - i];
        out[len - 1 - i] = t;
    }
    for (int j = 0; j < ORC_LANES; j++) states[j] = (uint32_t)x[j];
    *out_len = len;
    return ORC_OK;
}

/*
 * Interleaved rANS decoder, the plain definition: symbols in increasing
 * order, symbol i on state i mod 32.  slot = x mod 4096; s is the symbol with
 * c_s <= slot < c_s + f_s (linear scan); x <- f_s * floor(x / 4096) + slot -
 * c_s; while x < L, x <- 256 x + next byte.  Every state must enter in
 * [L, 2^31) and end at exactly L, and every byte must be consumed.
 */
int oracle_rans_decode(const uint8_t *bytes, uint32_t nbytes, const uint32_t states[32],
                       const uint16_t freq[256], uint32_t n, uint8_t *sym)
{
    uint32_t cum[257];
    cumulative(freq, cum);
    if (n > 0 && cum[256] != ORC_M) return ORC_E_CORRUPT;
    uint64_t x[ORC_LANES];
    for (int j = 0; j < ORC_LANES; j++) {
        x[j] = states[j];
        if (n > 0 && (x[j] < ORC_L || x[j] >= (1ULL << 31))) return ORC_E_CORRUPT;
    }
    uint32_t pos = 0;
    for (uint32_t k = 0; k < n; k++) {
        uint64_t *xs = &x[k % ORC_LANES];
        uint32_t slot = (uint32_t)(*xs % ORC_M);
        uint32_t s = 0;
        while (!(cum[s] <= slot && slot < cum[s] + freq[s])) s++;
        sym[k] = (uint8_t)s;
        *xs = freq[s] * (*xs / ORC_M) + slot - cum[s];
        while (*xs < ORC_L) {
            if (pos >= nbytes) return ORC_E_CORRUPT;
            *xs = (*xs << 8) | bytes[pos++];
        }
    }
    if (pos != nbytes) return ORC_E_CORRUPT;
    if (n > 0)
        for (int j = 0; j < ORC_LANES; j++)
            if (x[j] != ORC_L) return ORC_E_CORRUPT;
    return ORC_OK;
}

/* ------------------------------------------------------------ LZ parse */

typedef struct {
    uint32_t lit_run, match_len;
    uint64_t src;
} token;

typedef struct {
    token *tok;
    uint32_t ntok, cap;
} token_list;

static int push_token(token_list *tl, uint32_t lit_run, uint32_t match_len, uint64_t src)
{
    if (tl->ntok == tl->cap) {
        uint32_t nc = tl->cap ? 2 * tl->cap : 64;
        token *t = realloc(tl->tok, nc * sizeof(token));
        if (!t) return ORC_E_NOMEM;
        tl->tok = t;
        tl->cap = nc;
    }
    tl->tok[tl->ntok].lit_run = lit_run;
    tl->tok[tl->ntok].match_len = match_len;
    tl->tok[tl->ntok].src = src;
    tl->ntok++;
    return ORC_OK;
}

static uint32_t hash4(const uint8_t *p)
{
    uint32_t v = (uint32_t)p[0] | (uint32_t)p[1] << 8 | (uint32_t)p[2] << 16 | (uint32_t)p[3] << 24;
    return (v * 2654435761u) >> 12; /* 20-bit bucket */
}

/*
 * Greedy global match search (Section 2): at each position p, the longest
 * earlier occurrence q < p (anywhere in the file, overlap with p allowed)
 * among the candidates sharing p's first four bytes, walked most recent
 * first (all of them when max_chain is 0); ties go to the smaller q.  A match
 * of at least min_match bytes is taken, its destination clipped at the end of
 * p's block; otherwise p is a literal.  Each block ends with a token whose
 * match length is 0.
 */
static int lz_parse(const uint8_t *in, uint64_t n, uint64_t B, uint32_t min_match,
                    uint32_t max_chain, token_list *blocks, uint64_t nb)
{
    const uint32_t NH = 1u << 20;
    int64_t *head = malloc(NH * sizeof(int64_t));
    int64_t *prev = malloc((n ? n : 1) * sizeof(int64_t));
    if (!head || !prev) { free(head); free(prev); return ORC_E_NOMEM; }
    for (uint32_t i = 0; i < NH; i++) head[i] = -1;
    uint64_t inserted = 0; /* positions [0, inserted) are in the chains */
    for (uint64_t b = 0; b < nb; b++) {
        uint64_t bstart = b * B, bend = bstart + B < n ? bstart + B : n;
        uint64_t p = bstart;
        uint32_t lit = 0;
        while (p < bend) {
            while (inserted < p) { /* chains hold exactly the positions before p */
                if (inserted + 4 <= n) {
                    uint32_t h = hash4(in + inserted);
                    prev[inserted] = head[h];
                    head[h] = (int64_t)inserted;
                }
                inserted++;
            }
            uint64_t best_len = 0, best_q = 0;
            if (bend - p >= min_match && p + 4 <= n) {
                uint32_t depth = 0;
                for (int64_t q = head[hash4(in + p)]; q >= 0; q = prev[q]) {
                    if (max_chain && depth++ >= max_chain) break;
                    uint64_t l = 0;
                    while (p + l < bend && in[q + l] == in[p + l]) l++;
                    if (l > best_len || (l == best_len && l > 0 && (uint64_t)q < best_q)) {
                        best_len = l;
                        best_q = (uint64_t)q;
                    }
                }
            }
            if (best_len >= min_match) {
                if (push_token(&blocks[b], lit, (uint32_t)best_len, best_q)) { free(head); free(prev); return ORC_E_NOMEM; }
                lit = 0;
                p += best_len;
            } else {
                lit++;
                p++;
            }
        }
        if (push_token(&blocks[b], lit, 0, 0)) { free(head); free(prev); return ORC_E_NOMEM; }
    }
    free(head);
    free(prev);
    return ORC_OK;
}

/* ------------------------------------------------------ stream encoding */

typedef struct {
    uint8_t *d;
    uint32_t n, cap;
} bytes_t;

static int put(bytes_t *b, uint8_t v)
{
    if (b->n == b->cap) {
        uint32_t nc = b->cap ? 2 * b->cap : 256;
        uint8_t *t = realloc(b->d, nc);
        if (!t) return ORC_E_NOMEM;
        b->d = t;
        b->cap = nc;
    }
    b->d[b->n++] = v;
    return ORC_OK;
}

/* entropy-code one stream into dst (16-byte aligned position), returning its byte count */
static int write_stream(const uint8_t *sym, uint32_t n, uint8_t *dst, uint64_t cap, uint64_t *nbytes)
{
    if (n == 0) { *nbytes = 0; return ORC_OK; }
    uint16_t freq[256];
    oracle_rans_freqs(sym, n, freq);
    uint32_t present = 0;
    for (int s = 0; s < 256; s++) present += freq[s] != 0;
    uint64_t head = 128 + 32 + align16(2ull * present);
    if (head > cap) return ORC_E_NOMEM;
    uint32_t states[32], rlen = 0;
    int rc = oracle_rans_encode(sym, n, freq, states, dst + head, (uint32_t)(cap - head), &rlen);
    if (rc) return rc;
    for (int j = 0; j < 32; j++) wr(dst + 4 * j, states[j], 4);
    memset(dst + 128, 0, 32);
    uint64_t fo = 160;
    for (int s = 0; s < 256; s++) {
        if (!freq[s]) continue;
        dst[128 + s / 8] |= (uint8_t)(1u << (s % 8));
        wr(dst + fo, freq[s], 2);
        fo += 2;
    }
    while (fo < head) dst[fo++] = 0;
    *nbytes = head + rlen;
    return ORC_OK;
}

static int cmp_range(const void *a, const void *b)
{
    const uint64_t *x = a, *y = b;
    return x[0] < y[0] ? -1 : x[0] > y[0] ? 1 : (x[1] < y[1] ? -1 : x[1] > y[1]);
}

uint64_t oracle_encode_bound(uint64_t n, uint32_t log2_block)
{
    uint64_t B = 1ull << log2_block, nb = (n + B - 1) / B;
    return 64 + 16 + nb * (9 * B + 4096);
}

/*
 * Whole-archive encoder.  Parses with the greedy global search, separates
 * each block's tokens into the literal, length and absolute-offset streams
 * (Section 2, "stream separation"), entropy-codes each stream of each block
 * on its own (Section 3), and records per block the earlier blocks its
 * matches read (Section 2: a block decodes once the blocks holding its source
 * bytes are present).
 */
int oracle_encode(const uint8_t *in, uint64_t n, uint32_t log2_block, uint32_t min_match,
                  uint32_t max_chain, uint8_t *arc, uint64_t cap, uint64_t *arc_len)
{
    return oracle_encode_adaptive(in, n, log2_block, min_match, max_chain, 0, arc, cap, arc_len);
}

/*
 * As oracle_encode; with adaptive set, each stream of each block is stored
 * verbatim (mode 1) when its rANS coding would take at least as many bytes
 * as its symbols (Section 4: whether entropy coding pays is data-dependent,
 * so it is decided per stream at encode time).
 */
int oracle_encode_adaptive(const uint8_t *in, uint64_t n, uint32_t log2_block, uint32_t min_match,
                           uint32_t max_chain, uint32_t adaptive, uint8_t *arc, uint64_t cap,
                           uint64_t *arc_len)
{
    if (log2_block < 8 || log2_block > 16 || min_match < 4) return ORC_E_INVAL;
    uint64_t B = 1ull << log2_block, nb = (n + B - 1) / B;
    int w = n > (1ull << 32) ? 5 : 4;
    if (cap < oracle_encode_bound(n, log2_block)) return ORC_E_NOMEM;
    token_list *blocks = calloc(nb ? nb : 1, sizeof(token_list));
    if (!blocks) return ORC_E_NOMEM;
    int rc = lz_parse(in, n, B, min_match, max_chain, blocks, nb);

    /* dependency intervals per block: the earlier blocks each match reads */
    uint32_t *dep_ptr = calloc(nb + 1, sizeof(uint32_t));
    uint64_t iv_cap = 1024, niv = 0;
    uint32_t *iv = malloc(iv_cap * 2 * sizeof(uint32_t));
    if (!dep_ptr || !iv) rc = ORC_E_NOMEM;
    for (uint64_t b = 0; rc == ORC_OK && b < nb; b++) {
        uint64_t dst = b * B;
        uint32_t nr = 0;
        uint64_t *rg = malloc(2 * sizeof(uint64_t) * (blocks[b].ntok + 1));
        if (!rg) { rc = ORC_E_NOMEM; break; }
        for (uint32_t t = 0; t < blocks[b].ntok; t++) {
            token *tk = &blocks[b].tok[t];
            dst += tk->lit_run;
            if (tk->match_len) {
                uint64_t rl = tk->match_len < dst - tk->src ? tk->match_len : dst - tk->src;
                uint64_t f = tk->src / B, l = (tk->src + rl - 1) / B;
                if (l >= b) l = b - 1; /* bytes inside the block itself are no dependency */
                if (f <= l && f < b) { rg[2 * nr] = f; rg[2 * nr + 1] = l; nr++; }
            }
            dst += tk->match_len;
        }
        qsort(rg, nr, 2 * sizeof(uint64_t), cmp_range);
        dep_ptr[b] = (uint32_t)niv;
        for (uint32_t i = 0; i < nr && rc == ORC_OK;) {
            uint64_t f = rg[2 * i], l = rg[2 * i + 1];
            uint32_t j = i + 1;
            while (j < nr && rg[2 * j] <= l + 1) { /* merge overlapping or adjacent runs */
                if (rg[2 * j + 1] > l) l = rg[2 * j + 1];
                j++;
            }
            if (niv == iv_cap) {
                iv_cap *= 2;
                uint32_t *t2 = realloc(iv, iv_cap * 2 * sizeof(uint32_t));
                if (!t2) { rc = ORC_E_NOMEM; break; }
                iv = t2;
            }
            iv[2 * niv] = (uint32_t)f;
            iv[2 * niv + 1] = (uint32_t)l;
            niv++;
            i = j;
        }
        free(rg);
    }
    if (rc == ORC_OK) dep_ptr[nb] = (uint32_t)niv;

    uint64_t dir_off = ORC_HDR, deps_off = dir_off + ORC_DIR * nb;
    uint64_t payload_off = align16(deps_off + 4 * (nb + 1) + 8 * niv);
    uint64_t pos = payload_off;
    if (rc == ORC_OK) memset(arc, 0, payload_off);
    for (uint64_t b = 0; rc == ORC_OK && b < nb; b++) {
        token_list *tl = &blocks[b];
        bytes_t lit = {0}, esc = {0}, codes = {0}, off = {0};
        uint64_t dst = b * B;
        const uint8_t *base = in;
        for (uint32_t t = 0; t < tl->ntok && rc == ORC_OK; t++) {
            token *tk = &tl->tok[t];
            for (uint32_t i = 0; i < tk->lit_run; i++) rc |= put(&lit, base[dst + i]);
            uint32_t v2[2] = {tk->lit_run, tk->match_len};
            for (int k = 0; k < 2; k++) {
                if (v2[k] < 255) {
                    rc |= put(&codes, (uint8_t)v2[k]);
                } else {
                    rc |= put(&codes, 255);
                    rc |= put(&esc, (uint8_t)((v2[k] - 255) & 0xff));
                    rc |= put(&esc, (uint8_t)((v2[k] - 255) >> 8));
                }
            }
            if (t + 1 < tl->ntok)
                for (int k = 0; k < w; k++) rc |= put(&off, (uint8_t)(tk->src >> (8 * k)));
            dst += tk->lit_run + tk->match_len;
        }
        /* length stream = escape values, then the codes */
        bytes_t lens = {0};
        for (uint32_t i = 0; i < esc.n && rc == ORC_OK; i++) rc |= put(&lens, esc.d[i]);
        for (uint32_t i = 0; i < codes.n && rc == ORC_OK; i++) rc |= put(&lens, codes.d[i]);
        uint8_t *dir = arc + dir_off + ORC_DIR * b;
        const bytes_t *st[3] = {&lit, &lens, &off};
        for (int k = 0; k < ORC_NSTREAM && rc == ORC_OK; k++) {
            uint64_t nbytes = 0;
            pos = align16(pos);
            rc = write_stream(st[k]->d, st[k]->n, arc + pos, cap - pos, &nbytes);
            uint8_t mode = 0; /* rANS */
            if (rc == ORC_OK && adaptive && st[k]->n && nbytes >= st[k]->n) {
                memcpy(arc + pos, st[k]->d, st[k]->n); /* stored: rANS did not shrink it */
                memset(arc + pos + st[k]->n, 0, nbytes - st[k]->n);
                nbytes = st[k]->n;
                mode = 1;
            }
            wr(dir + 8 * k, pos - payload_off, 8);
            wr(dir + 24 + 4 * k, nbytes, 4);
            wr(dir + 36 + 4 * k, st[k]->n, 4);
            dir[56 + k] = mode;
            pos += nbytes;
        }
        wr(dir + 48, tl->ntok, 4);
        wr(dir + 52, esc.n / 2, 4);
        free(lit.d); free(esc.d); free(codes.d); free(off.d); free(lens.d);
    }
    if (rc == ORC_OK) {
        pos = align16(pos);
        memcpy(arc, "ACEA", 4);
        wr(arc + 4, 1, 2);
        arc[6] = ORC_NSTREAM;
        arc[7] = ORC_LANES;
        arc[8] = ORC_SCALE_BITS;
        arc[9] = (uint8_t)w;
        arc[10] = (uint8_t)log2_block;
        arc[11] = 0;
        wr(arc + 12, 0, 4);
        wr(arc + 16, n, 8);
        wr(arc + 24, nb, 8);
        wr(arc + 32, dir_off, 8);
        wr(arc + 40, deps_off, 8);
        wr(arc + 48, payload_off, 8);
        wr(arc + 56, pos, 8);
        for (uint64_t b = 0; b <= nb; b++) wr(arc + deps_off + 4 * b, dep_ptr[b], 4);
        for (uint64_t i = 0; i < 2 * niv; i++) wr(arc + deps_off + 4 * (nb + 1) + 4 * i, iv[i], 4);
        *arc_len = pos;
    }
    for (uint64_t b = 0; b < nb; b++) free(blocks[b].tok);
    free(blocks); free(dep_ptr); free(iv);
    return rc;
}

/* ------------------------------------------------------------- reading */

typedef struct {
    uint64_t total, nb, dir_off, deps_off, payload_off, arc_bytes;
    uint32_t B;
    int w;
} header_t;

static int read_header(const uint8_t *arc, uint64_t arc_len, header_t *h)
{
    if (arc_len < ORC_HDR || memcmp(arc, "ACEA", 4) != 0) return ORC_E_CORRUPT;
    if (rd(arc + 4, 2) != 1 || arc[6] != ORC_NSTREAM || arc[7] != ORC_LANES ||
        arc[8] != ORC_SCALE_BITS)
        return ORC_E_CORRUPT;
    h->w = arc[9];
    if (h->w != 4 && h->w != 5) return ORC_E_CORRUPT;
    if (arc[10] < 8 || arc[10] > 16) return ORC_E_CORRUPT;
    h->B = 1u << arc[10];
    h->total = rd(arc + 16, 8);
    h->nb = rd(arc + 24, 8);
    h->dir_off = rd(arc + 32, 8);
    h->deps_off = rd(arc + 40, 8);
    h->payload_off = rd(arc + 48, 8);
    h->arc_bytes = rd(arc + 56, 8);
    if (h->nb != (h->total + h->B - 1) / h->B) return ORC_E_CORRUPT;
    if (h->arc_bytes > arc_len || h->payload_off > h->arc_bytes) return ORC_E_CORRUPT;
    if (h->dir_off + ORC_DIR * h->nb > h->deps_off) return ORC_E_CORRUPT;
    if (h->deps_off + 4 * (h->nb + 1) > h->payload_off) return ORC_E_CORRUPT;
    return ORC_OK;
}

int oracle_info(const uint8_t *arc, uint64_t arc_len, uint64_t *total, uint32_t *block_size,
                uint64_t *n_blocks, uint32_t *off_width)
{
    header_t h;
    int rc = read_header(arc, arc_len, &h);
    if (rc) return rc;
    *total = h.total;
    *block_size = h.B;
    *n_blocks = h.nb;
    *off_width = (uint32_t)h.w;
    return ORC_OK;
}

/* rANS-decode stream k of block b into a fresh buffer of nsym symbols */
static int read_stream(const uint8_t *arc, const header_t *h, uint64_t b, int k,
                       uint8_t **sym_out, uint32_t *nsym_out)
{
    const uint8_t *dir = arc + h->dir_off + ORC_DIR * b;
    uint64_t off = h->payload_off + rd(dir + 8 * k, 8);
    uint32_t nbytes = (uint32_t)rd(dir + 24 + 4 * k, 4);
    uint32_t n = (uint32_t)rd(dir + 36 + 4 * k, 4);
    const uint8_t mode = dir[56 + k];
    if (mode > 1) return ORC_E_CORRUPT; /* 0: rANS, 1: stored */
    uint8_t *sym = malloc(n ? n : 1);
    if (!sym) return ORC_E_NOMEM;
    *sym_out = sym;
    *nsym_out = n;
    if (n == 0) return nbytes == 0 ? ORC_OK : ORC_E_CORRUPT;
    if (mode == 1) { /* stored: the bytes are the symbols */
        if (nbytes != n || off + nbytes > h->arc_bytes) return ORC_E_CORRUPT;
        memcpy(sym, arc + off, n);
        return ORC_OK;
    }
    if (off + nbytes > h->arc_bytes || nbytes < 160) return ORC_E_CORRUPT;
    const uint8_t *p = arc + off;
    uint32_t states[32];
    for (int j = 0; j < 32; j++) states[j] = (uint32_t)rd(p + 4 * j, 4);
    uint16_t freq[256];
    uint32_t present = 0;
    for (int s = 0; s < 256; s++) present += (p[128 + s / 8] >> (s % 8)) & 1;
    uint64_t head = 160 + align16(2ull * present);
    if (head > nbytes) return ORC_E_CORRUPT;
    uint32_t fi = 0;
    for (int s = 0; s < 256; s++) {
        freq[s] = 0;
        if ((p[128 + s / 8] >> (s % 8)) & 1) {
            freq[s] = (uint16_t)rd(p + 160 + 2 * fi, 2);
            fi++;
            if (freq[s] == 0) return ORC_E_CORRUPT;
        }
    }
    return oracle_rans_decode(p + head, (uint32_t)(nbytes - head), states, freq, n, sym);
}

/* decode the token list of block b (both layers' inputs, entropy layer undone) */
static int block_tokens(const uint8_t *arc, const header_t *h, uint64_t b, token_list *tl,
                        uint8_t **lit_out, uint32_t *nlit_out)
{
    uint8_t *s[3] = {0, 0, 0};
    uint32_t n[3] = {0, 0, 0};
    int rc = ORC_OK;
    for (int k = 0; k < 3 && rc == ORC_OK; k++) rc = read_stream(arc, h, b, k, &s[k], &n[k]);
    const uint8_t *dir = arc + h->dir_off + ORC_DIR * b;
    uint32_t ntok = (uint32_t)rd(dir + 48, 4), nesc = (uint32_t)rd(dir + 52, 4);
    if (rc == ORC_OK && ((uint64_t)n[S_LEN] != 2ull * nesc + 2ull * ntok ||
                         (uint64_t)n[S_OFF] != (uint64_t)h->w * (ntok ? ntok - 1 : 0) || ntok == 0))
        rc = ORC_E_CORRUPT;
    uint32_t e = 0;
    const uint8_t *codes = s[S_LEN] + 2 * (uint64_t)nesc;
    for (uint32_t t = 0; rc == ORC_OK && t < ntok; t++) {
        uint32_t v[2];
        for (int k = 0; k < 2; k++) {
            uint8_t c = codes[2 * t + k];
            if (c < 255) {
                v[k] = c;
            } else {
                if (e >= nesc) { rc = ORC_E_CORRUPT; break; }
                v[k] = 255 + (uint32_t)rd(s[S_LEN] + 2 * e, 2);
                e++;
            }
        }
        if (rc) break;
        uint64_t src = t + 1 < ntok ? rd(s[S_OFF] + (uint64_t)h->w * t, h->w) : 0;
        rc = push_token(tl, v[0], v[1], src);
    }
    if (rc == ORC_OK && e != nesc) rc = ORC_E_CORRUPT;
    free(s[S_LEN]);
    free(s[S_OFF]);
    if (rc) { free(s[S_LIT]); return rc; }
    *lit_out = s[S_LIT];
    *nlit_out = n[S_LIT];
    return ORC_OK;
}

/*
 * Decode block b into image, whose byte i is absolute output position i.
 * Literals are appended in order; a match copies byte by byte from its
 * absolute source, so a source overlapping its own destination repeats, as
 * in sequential LZ77 (Section 2, Section 3).
 */
static int decode_block(const uint8_t *arc, const header_t *h, uint64_t b, uint8_t *image)
{
    token_list tl = {0};
    uint8_t *lit = NULL;
    uint32_t nlit = 0;
    int rc = block_tokens(arc, h, b, &tl, &lit, &nlit);
    if (rc) { free(tl.tok); return rc; }
    uint64_t bstart = b * (uint64_t)h->B;
    uint64_t bend = bstart + h->B < h->total ? bstart + h->B : h->total;
    uint64_t dst = bstart;
    uint32_t lp = 0;
    for (uint32_t t = 0; t < tl.ntok && rc == ORC_OK; t++) {
        token *tk = &tl.tok[t];
        if (tk->lit_run > nlit - lp || dst + tk->lit_run > bend) { rc = ORC_E_CORRUPT; break; }
        for (uint32_t i = 0; i < tk->lit_run; i++) image[dst++] = lit[lp++];
        if (tk->match_len) {
            if (tk->src >= dst || dst + tk->match_len > bend) { rc = ORC_E_CORRUPT; break; }
            for (uint32_t i = 0; i < tk->match_len; i++) image[dst + i] = image[tk->src + i];
            dst += tk->match_len;
        }
    }
    if (rc == ORC_OK && (dst != bend || lp != nlit)) rc = ORC_E_CORRUPT;
    free(tl.tok);
    free(lit);
    return rc;
}

int oracle_decode(const uint8_t *arc, uint64_t arc_len, uint8_t *out, uint64_t out_cap)
{
    header_t h;
    int rc = read_header(arc, arc_len, &h);
    if (rc) return rc;
    if (out_cap < h.total) return ORC_E_NOMEM;
    for (uint64_t b = 0; b < h.nb; b++)
        if ((rc = decode_block(arc, &h, b, out))) return rc;
    return ORC_OK;
}

int oracle_decode_block_tokens(const uint8_t *arc, uint64_t arc_len, uint64_t block,
                               uint32_t *lit_run, uint32_t *match_len, uint64_t *src,
                               uint32_t cap, uint32_t *ntok)
{
    header_t h;
    int rc = read_header(arc, arc_len, &h);
    if (rc) return rc;
    if (block >= h.nb) return ORC_E_RANGE;
    token_list tl = {0};
    uint8_t *lit = NULL;
    uint32_t nlit = 0;
    rc = block_tokens(arc, &h, block, &tl, &lit, &nlit);
    free(lit);
    if (rc == ORC_OK) {
        *ntok = tl.ntok;
        if (tl.ntok > cap) rc = ORC_E_NOMEM;
        for (uint32_t t = 0; rc == ORC_OK && t < tl.ntok; t++) {
            lit_run[t] = tl.tok[t].lit_run;
            match_len[t] = tl.tok[t].match_len;
            src[t] = tl.tok[t].src;
        }
    }
    free(tl.tok);
    return rc;
}

/* ------------------------------------------------ dependencies and seek */

static int deps_of(const uint8_t *arc, const header_t *h, uint64_t b, uint32_t *lo, uint32_t *hi)
{
    const uint8_t *d = arc + h->deps_off;
    *lo = (uint32_t)rd(d + 4 * b, 4);
    *hi = (uint32_t)rd(d + 4 * (b + 1), 4);
    if (*lo > *hi || h->deps_off + 4 * (h->nb + 1) + 8ull * *hi > h->payload_off) return ORC_E_CORRUPT;
    return ORC_OK;
}

static void interval(const uint8_t *arc, const header_t *h, uint32_t i, uint64_t *first, uint64_t *last)
{
    const uint8_t *p = arc + h->deps_off + 4 * (h->nb + 1) + 8ull * i;
    *first = rd(p, 4);
    *last = rd(p + 4, 4);
}

/* level[b] = 0 without sources in other blocks, else 1 + the largest level among them */
int oracle_levels(const uint8_t *arc, uint64_t arc_len, uint32_t *level)
{
    header_t h;
    int rc = read_header(arc, arc_len, &h);
    if (rc) return rc;
    for (uint64_t b = 0; b < h.nb; b++) {
        uint32_t lo, hi, lv = 0;
        if ((rc = deps_of(arc, &h, b, &lo, &hi))) return rc;
        for (uint32_t i = lo; i < hi; i++) {
            uint64_t f, l;
            interval(arc, &h, i, &f, &l);
            if (f > l || l >= b) return ORC_E_CORRUPT;
            for (uint64_t k = f; k <= l; k++)
                if (level[k] + 1 > lv) lv = level[k] + 1;
        }
        level[b] = lv;
    }
    return ORC_OK;
}

/* mark the blocks [first, last] and every block their matches read, transitively */
int oracle_closure(const uint8_t *arc, uint64_t arc_len, uint64_t first, uint64_t last,
                   uint8_t *in_closure)
{
    header_t h;
    int rc = read_header(arc, arc_len, &h);
    if (rc) return rc;
    if (first > last || last >= h.nb) return ORC_E_RANGE;
    memset(in_closure, 0, h.nb);
    for (uint64_t b = first; b <= last; b++) in_closure[b] = 1;
    /* sources always precede, so one pass from the highest block down suffices */
    for (uint64_t b = last + 1; b-- > 0;) {
        if (!in_closure[b]) continue;
        uint32_t lo, hi;
        if ((rc = deps_of(arc, &h, b, &lo, &hi))) return rc;
        for (uint32_t i = lo; i < hi; i++) {
            uint64_t f, l;
            interval(arc, &h, i, &f, &l);
            if (f > l || l >= b) return ORC_E_CORRUPT;
            for (uint64_t k = f; k <= l; k++) in_closure[k] = 1;
        }
    }
    return ORC_OK;
}

/*
 * Unified seek (Section 5): the coordinate range [coord, coord+len) names
 * its covering blocks; those blocks and the blocks their matches read are
 * decoded from the archive alone into a scratch image, and only the
 * requested bytes are copied out.
 */
int oracle_seek(const uint8_t *arc, uint64_t arc_len, uint64_t coord, uint64_t len, uint8_t *out)
{
    header_t h;
    int rc = read_header(arc, arc_len, &h);
    if (rc) return rc;
    if (len == 0 || coord >= h.total || len > h.total - coord) return ORC_E_RANGE;
    uint8_t *in = malloc(h.nb);
    uint8_t *image = calloc(h.total, 1);
    if (!in || !image) { free(in); free(image); return ORC_E_NOMEM; }
    rc = oracle_closure(arc, arc_len, coord / h.B, (coord + len - 1) / h.B, in);
    for (uint64_t b = 0; rc == ORC_OK && b < h.nb; b++)
        if (in[b]) rc = decode_block(arc, &h, b, image);
    if (rc == ORC_OK) memcpy(out, image + coord, len);
    free(in);
    free(image);
    return rc;
}
