/*
 * Seeded synthetic inputs for the two-layer codec: the originals that the
 * codec compresses, plus the workload tables (object sizes, seek targets,
 * request streams) that drive it.
 *
 * This module holds no codec arithmetic at all: no entropy coding, no match
 * search, no archive layout.  Both the plain CPU oracle (through the tests)
 * and the GPU library's benchmark draw their inputs from here, so the two
 * sides see byte-identical data for a given seed.
 *
 * Every random draw comes from SplitMix64 (Steele, Lea, Flood, "Fast
 * splittable pseudorandom number generators", OOPSLA 2014): a 64-bit
 * counter advanced by the golden-gamma 0x9e3779b97f4a7c15 and finalised by
 * two xor-shift-multiply rounds.  Floating point is used only through
 * +, -, *, / and the deterministic log/exp below (this file is compiled with
 * -ffp-contract=off), so the same seed gives the same bytes on x86-64 and on
 * aarch64.
 *
 * The shapes follow the paper's four data profiles (Section 6, Table 1:
 * FASTQ reads, a repetitive genome, English text, mixed data); the real data
 * sets are not available, so these generators stand in for them.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <stdio.h>

/* ------------------------------------------------------------------ RNG */

static inline uint64_t sm64_next(uint64_t *s)
{
    uint64_t z = (*s += 0x9e3779b97f4a7c15ULL);
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

/* uniform integer in [lo, hi] (inclusive), by 64x64->128 multiply-high */
static inline uint64_t sm64_range(uint64_t *s, uint64_t lo, uint64_t hi)
{
    uint64_t span = hi - lo + 1;
    if (span == 0) return sm64_next(s); /* full 64-bit range */
    return lo + (uint64_t)(((unsigned __int128)sm64_next(s) * span) >> 64);
}

/* uniform double in [0, 1) with 53 random bits */
static inline double sm64_unit(uint64_t *s)
{
    return (double)(sm64_next(s) >> 11) * (1.0 / 9007199254740992.0);
}

uint64_t synth_splitmix64(uint64_t *state) { return sm64_next(state); }

/* ------------------------------------------- deterministic log and exp */

static const double LN2 = 0.69314718055994530942;

/* natural log for x > 0: x = m * 2^e with m in [1,2), ln m = 2 atanh((m-1)/(m+1)) */
static double det_log(double x)
{
    int e = 0;
    double m = x;
    while (m >= 2.0) { m *= 0.5; e++; }
    while (m < 1.0) { m *= 2.0; e--; }
    double t = (m - 1.0) / (m + 1.0), t2 = t * t, term = t, sum = 0.0;
    for (int k = 1; k < 80; k += 2) {
        sum += term / (double)k;
        term *= t2;
    }
    return 2.0 * sum + (double)e * LN2;
}

/* e^x: x = k ln2 + r, r in [0, ln2), Taylor series for e^r, scale by 2^k */
static double det_exp(double x)
{
    double kf = x / LN2;
    long k = (long)kf;
    if ((double)k > kf) k--; /* floor */
    double r = x - (double)k * LN2, term = 1.0, sum = 1.0;
    for (int n = 1; n < 30; n++) {
        term = term * r / (double)n;
        sum += term;
    }
    while (k > 0) { sum *= 2.0; k--; }
    while (k < 0) { sum *= 0.5; k++; }
    return sum;
}

double synth_det_log(double x) { return det_log(x); }
double synth_det_exp(double x) { return det_exp(x); }

/* floor(exp(U[ln lo, ln hi])): a log-uniform integer in [lo, hi] */
static uint64_t log_uniform(uint64_t *s, uint64_t lo, uint64_t hi)
{
    double a = det_log((double)lo), b = det_log((double)hi);
    double v = det_exp(a + (b - a) * sm64_unit(s));
    uint64_t r = (uint64_t)v;
    if (r < lo) r = lo;
    if (r > hi) r = hi;
    return r;
}

/* ------------------------------------------------------------- mixed/text */

#define VOCAB 5000
#define ZIPF_S 1.1

/*
 * Mixed profile.  A vocabulary of 5,000 distinct words (length U[2,10],
 * letters uniform a-z); words are emitted with Zipf(s = 1.1) rank
 * probabilities, each followed by a space.  While fewer than copy_frac of
 * the bytes written so far came from copies (and at least 512 bytes exist),
 * a copy of an earlier span of U[32,512] bytes, starting at a uniform earlier
 * absolute offset and not overlapping its destination, is appended instead.
 * copy_frac = 0 gives the text profile.  Output is truncated at n bytes.
 */
uint64_t synth_mixed(uint8_t *out, uint64_t n, uint64_t seed, double copy_frac)
{
    uint64_t s = seed;
    char (*words)[11] = calloc(VOCAB, sizeof *words);
    uint8_t *wlen = calloc(VOCAB, 1);
    double *cdf = calloc(VOCAB, sizeof *cdf);
    /* open-addressing set of word hashes to keep words distinct */
    const uint32_t HS = 1u << 15;
    uint64_t *hset = calloc(HS, sizeof *hset);
    if (!words || !wlen || !cdf || !hset) { free(words); free(wlen); free(cdf); free(hset); return 0; }
    int nw = 0;
    while (nw < VOCAB) {
        int len = (int)sm64_range(&s, 2, 10);
        char w[11];
        uint64_t h = 1469598103934665603ULL; /* string key for the distinctness set */
        for (int i = 0; i < len; i++) {
            w[i] = (char)('a' + sm64_range(&s, 0, 25));
            h = (h ^ (uint8_t)w[i]) * 1099511628211ULL;
        }
        h = (h ^ (uint64_t)len) | 1; /* never zero: zero marks an empty slot */
        uint32_t slot = (uint32_t)(h & (HS - 1));
        int dup = 0;
        while (hset[slot]) {
            if (hset[slot] == h) { dup = 1; break; }
            slot = (slot + 1) & (HS - 1);
        }
        if (dup) continue; /* equal key: treat as a duplicate word and redraw */
        hset[slot] = h;
        memcpy(words[nw], w, (size_t)len);
        wlen[nw] = (uint8_t)len;
        nw++;
    }
    double total = 0.0;
    for (int k = 0; k < VOCAB; k++) {
        total += det_exp(-ZIPF_S * det_log((double)(k + 1)));
        cdf[k] = total;
    }
    for (int k = 0; k < VOCAB; k++) cdf[k] /= total;

    uint64_t pos = 0, copied = 0;
    while (pos < n) {
        if (pos >= 512 && (double)copied < copy_frac * (double)pos) {
            uint64_t len = sm64_range(&s, 32, 512);
            uint64_t src = sm64_range(&s, 0, pos - len);
            for (uint64_t i = 0; i < len && pos < n; i++) out[pos++] = out[src + i];
            copied += len;
        } else {
            double u = sm64_unit(&s);
            int lo = 0, hi = VOCAB - 1;
            while (lo < hi) { /* first rank whose cdf exceeds u */
                int mid = (lo + hi) / 2;
                if (cdf[mid] > u) hi = mid; else lo = mid + 1;
            }
            for (int i = 0; i < wlen[lo] && pos < n; i++) out[pos++] = (uint8_t)words[lo][i];
            if (pos < n) out[pos++] = ' ';
        }
    }
    free(words); free(wlen); free(cdf); free(hset);
    return pos;
}

/* ------------------------------------------------------------------ FASTQ */

/*
 * FASTQ profile.  Records "@SIM:1:FC:<lane>:<tile>:<x>:<y>\n<150 bases>\n+\n
 * <150 quality>\n".  y grows by U[1,20] per record; past 99999 it restarts at
 * U[1,20] and x grows by one; tile starts at 1101 and grows every 10^6
 * records; lane (1..8) grows every 4 tiles.  Bases follow an order-2 Markov
 * chain over ACGT whose 16 transition rows are Dirichlet(1,1,1,1) draws
 * (uniform spacings); a base becomes N with probability 0.001.  Quality i is
 * round(N(mu_i, 3)) clipped to [2, 41] with mu_i falling linearly from 38 to
 * 28; the normal is the Irwin-Hall sum of 12 uniforms minus 6 (exact mean and
 * variance).  N gets quality 2.  Characters are quality + 33.
 */
uint64_t synth_fastq(uint8_t *out, uint64_t n, uint64_t seed)
{
    static const char ACGT[4] = {'A', 'C', 'G', 'T'};
    uint64_t s = seed;
    double cum[16][4];
    for (int c = 0; c < 16; c++) {
        double u[3] = {sm64_unit(&s), sm64_unit(&s), sm64_unit(&s)};
        for (int i = 0; i < 3; i++) /* sort three values */
            for (int j = i + 1; j < 3; j++)
                if (u[j] < u[i]) { double t = u[i]; u[i] = u[j]; u[j] = t; }
        cum[c][0] = u[0]; cum[c][1] = u[1]; cum[c][2] = u[2]; cum[c][3] = 2.0;
    }
    unsigned ctx = (unsigned)sm64_range(&s, 0, 15);
    uint64_t pos = 0, rec = 0, x = 1000, y = 0;
    char line[256];
    uint8_t qual[150];
    while (pos < n) {
        y += sm64_range(&s, 1, 20);
        if (y > 99999) { y = sm64_range(&s, 1, 20); x++; }
        uint64_t tile_idx = rec / 1000000;
        unsigned lane = 1 + (unsigned)((tile_idx / 4) % 8);
        unsigned tile = 1101 + (unsigned)tile_idx;
        int hl = snprintf(line, sizeof line, "@SIM:1:FC:%u:%u:%llu:%llu\n", lane, tile,
                          (unsigned long long)x, (unsigned long long)y);
        for (int i = 0; i < hl && pos < n; i++) out[pos++] = (uint8_t)line[i];
        for (int i = 0; i < 150; i++) {
            double v = sm64_unit(&s);
            int b = 0;
            while (v >= cum[ctx][b]) b++;
            ctx = ((ctx << 2) | (unsigned)b) & 15u;
            int isn = sm64_next(&s) % 1000 == 0;
            if (pos < n) out[pos++] = (uint8_t)(isn ? 'N' : ACGT[b]);
            double z = 0.0;
            for (int k = 0; k < 3; k++) {
                uint64_t r = sm64_next(&s);
                for (int q = 0; q < 4; q++) z += (double)((r >> (16 * q)) & 0xffff) * (1.0 / 65536.0);
            }
            z -= 6.0;
            double mu = 38.0 - 10.0 * (double)i / 149.0;
            double qv = mu + 3.0 * z + 0.5;
            long qi = (long)qv;
            if ((double)qi > qv) qi--; /* floor */
            if (qi < 2) qi = 2;
            if (qi > 41) qi = 41;
            qual[i] = (uint8_t)((isn ? 2 : qi) + 33);
        }
        const char *mid = "\n+\n";
        for (int i = 0; i < 3 && pos < n; i++) out[pos++] = (uint8_t)mid[i];
        for (int i = 0; i < 150 && pos < n; i++) out[pos++] = qual[i];
        if (pos < n) out[pos++] = '\n';
        rec++;
    }
    return pos;
}

/* ----------------------------------------------------------------- genome */

#define GENOME_BASE 1000000

/*
 * Repetitive genome profile.  A uniform random ACGT base sequence of 10^6
 * bases is written first; then, alternately, a tandem region (a random unit
 * of period U[2,50] repeated U[10,200] times) and a mutated copy of the base
 * sequence (each base: with p = 10^-3 a SNP to a different base chosen
 * uniformly, with p = 10^-4 an indel of length U[1,5], insertion or deletion
 * with equal odds).  No newlines.  Truncated at n bytes.
 */
uint64_t synth_genome(uint8_t *out, uint64_t n, uint64_t seed)
{
    static const char ACGT[4] = {'A', 'C', 'G', 'T'};
    uint64_t s = seed;
    uint8_t *base = malloc(GENOME_BASE);
    if (!base) return 0;
    for (int i = 0; i < GENOME_BASE; i += 32) {
        uint64_t r = sm64_next(&s);
        for (int j = 0; j < 32 && i + j < GENOME_BASE; j++) base[i + j] = (uint8_t)ACGT[(r >> (2 * j)) & 3];
    }
    uint64_t pos = 0;
    for (int i = 0; i < GENOME_BASE && pos < n; i++) out[pos++] = base[i];
    while (pos < n) {
        int period = (int)sm64_range(&s, 2, 50);
        int copies = (int)sm64_range(&s, 10, 200);
        uint8_t unit[50];
        for (int i = 0; i < period; i++) unit[i] = (uint8_t)ACGT[sm64_range(&s, 0, 3)];
        for (int c = 0; c < copies && pos < n; c++)
            for (int i = 0; i < period && pos < n; i++) out[pos++] = unit[i];
        for (int i = 0; i < GENOME_BASE && pos < n; i++) {
            uint64_t r = sm64_next(&s) >> 11; /* 53-bit uniform integer */
            const uint64_t P_SNP = 9007199254741ULL;  /* 10^-3 * 2^53 */
            const uint64_t P_INDEL = 900719925474ULL; /* 10^-4 * 2^53 */
            if (r < P_SNP) {
                int b = 0;
                while (ACGT[b] != base[i]) b++;
                int nb = (b + 1 + (int)sm64_range(&s, 0, 2)) & 3;
                out[pos++] = (uint8_t)ACGT[nb];
            } else if (r < P_SNP + P_INDEL) {
                int len = (int)sm64_range(&s, 1, 5);
                if (sm64_next(&s) & 1) { /* insertion after this base */
                    out[pos++] = base[i];
                    for (int k = 0; k < len && pos < n; k++) out[pos++] = (uint8_t)ACGT[sm64_range(&s, 0, 3)];
                } else { /* deletion of len bases starting here */
                    i += len - 1;
                }
            } else {
                out[pos++] = base[i];
            }
        }
    }
    free(base);
    return pos;
}

/* ---------------------------------------------------------- dispatch */

enum { SYNTH_FASTQ = 0, SYNTH_GENOME = 1, SYNTH_TEXT = 2, SYNTH_MIXED = 3 };

uint64_t synth_profile(int profile, uint8_t *out, uint64_t n, uint64_t seed)
{
    switch (profile) {
    case SYNTH_FASTQ: return synth_fastq(out, n, seed);
    case SYNTH_GENOME: return synth_genome(out, n, seed);
    case SYNTH_TEXT: return synth_mixed(out, n, seed, 0.0);
    case SYNTH_MIXED: return synth_mixed(out, n, seed, 0.4);
    default: return 0;
    }
}

/* ------------------------------------------------------ workload tables */

/*
 * The uneven batch: count objects, size floor(exp(U[ln min, ln max])),
 * profile uniform over the four, block size uniform over {4, 16, 64} KiB,
 * per-object seed = seed_base + k.
 */
void synth_objects(uint64_t seed, uint32_t count, uint64_t min_size, uint64_t max_size,
                   uint64_t seed_base, uint64_t *sizes, int32_t *profiles,
                   uint32_t *block_sizes, uint64_t *seeds)
{
    static const uint32_t BS[3] = {4096, 16384, 65536};
    uint64_t s = seed;
    for (uint32_t k = 0; k < count; k++) {
        sizes[k] = log_uniform(&s, min_size, max_size);
        profiles[k] = (int32_t)sm64_range(&s, 0, 3);
        block_sizes[k] = BS[sm64_range(&s, 0, 2)];
        seeds[k] = seed_base + k;
    }
}

/* count uniform integers in [lo, hi] */
void synth_uniform(uint64_t seed, uint32_t count, uint64_t lo, uint64_t hi, uint64_t *out)
{
    uint64_t s = seed;
    for (uint32_t k = 0; k < count; k++) out[k] = sm64_range(&s, lo, hi);
}

/* count log-uniform integers in [lo, hi] */
void synth_log_uniform(uint64_t seed, uint32_t count, uint64_t lo, uint64_t hi, uint64_t *out)
{
    uint64_t s = seed;
    for (uint32_t k = 0; k < count; k++) out[k] = log_uniform(&s, lo, hi);
}

/*
 * A seek request stream: Poisson arrivals at rate per second (exponential
 * gaps, arrival times in ns), archive k chosen with probability proportional
 * to sizes[k], coordinate uniform in the archive, length log-uniform in
 * [len_lo, len_hi] clipped to the archive end.
 */
void synth_requests(uint64_t seed, uint32_t count, double rate, uint32_t n_archives,
                    const uint64_t *sizes, uint64_t len_lo, uint64_t len_hi,
                    uint64_t *t_ns, uint32_t *archive, uint64_t *coord, uint64_t *len)
{
    uint64_t s = seed, total = 0;
    for (uint32_t a = 0; a < n_archives; a++) total += sizes[a];
    double t = 0.0;
    for (uint32_t k = 0; k < count; k++) {
        double u = sm64_unit(&s);
        t += -det_log(1.0 - u) / rate * 1e9;
        t_ns[k] = (uint64_t)t;
        uint64_t pick = sm64_range(&s, 0, total - 1);
        uint32_t a = 0;
        while (pick >= sizes[a]) { pick -= sizes[a]; a++; }
        archive[k] = a;
        coord[k] = sm64_range(&s, 0, sizes[a] - 1);
        uint64_t l = log_uniform(&s, len_lo, len_hi);
        if (coord[k] + l > sizes[a]) l = sizes[a] - coord[k];
        len[k] = l;
    }
}
