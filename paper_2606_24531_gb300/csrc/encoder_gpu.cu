// GPU encoder of the two-layer codec: the whole encode on the device, from
// input bytes in device memory to an archive in device memory, in the byte
// layout of ace_format.h (the same format the host encoder writes and every
// decoder reads).
//
// Match layer (Section 2: greedy parse with a global match search, absolute
// back-references): candidates are found for every position at once, a
// thread per position -- the earliest earlier occurrence of the 16-byte keys
// around it (a table over the whole input, built with atomic minima) and
// the most recent repeats inside its block (hash chains built a warp per
// block) -- then one thread per block walks its positions greedily, taking
// at each the longest candidate allowed there.  Blocks are parsed in
// windows of 64 that take no sources from each other; the first three
// windows are parsed one after another, and every later block takes its
// external sources only from them, so dependency levels stay at most 3 as
// with the host encoder.  A match of a block's own earlier bytes resolves
// in waves (one reading only literals is wave 1, one reading wave-k bytes
// wave k + 1); candidates deeper than wave 3 are refused, and an external
// candidate nearly as long as the best is preferred.
// Entropy layer (Section 3): each block's literal, length and offset
// streams are rANS-coded, a warp per block, with 32 interleaved states,
// 12-bit frequencies quantised as the host encoder does, byte
// renormalisation; with the adaptive option a stream rANS would not shrink
// is stored (Section 6.1).
//
// The parse differs from the host encoder's (another valid archive of the
// same input); every decoder reads either.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <vector>

#include "ace.h"
#include "ace_device.cuh"
#include "ace_format.h"

using namespace ace;

namespace {

constexpr uint32_t kKey = 16;        // long-key length of the global table
constexpr uint32_t kStride = 8;      // positions whose keys enter the table
constexpr uint32_t kWin = 64;        // blocks of a parse window
constexpr uint32_t kHeadWins = 3;    // windows parsed one after another
constexpr uint32_t kHead = kWin * kHeadWins;
constexpr uint32_t kMaxWave = 3;     // deepest in-block resolution wave taken
constexpr uint32_t kCap = 32;        // match lengths measured by the candidate search (extended later)
constexpr uint32_t kHashBits4 = 12;  // in-block chains: hash of 4 bytes
constexpr uint64_t kEmpty = ~0ull;
constexpr uint32_t kMaxChain = 64;

__host__ __device__ inline uint64_t align16(uint64_t v) { return (v + 15) & ~15ull; }

__device__ __forceinline__ uint64_t ld64u(const uint8_t* p) {
  uint64_t v = 0;
#pragma unroll
  for (int k = 0; k < 8; k++) v |= (uint64_t)p[k] << (8 * k);
  return v;
}

__device__ __forceinline__ uint32_t ld32u(const uint8_t* p) {
  return (uint32_t)p[0] | ((uint32_t)p[1] << 8) | ((uint32_t)p[2] << 16) | ((uint32_t)p[3] << 24);
}

__device__ __forceinline__ uint32_t hash_key(const uint8_t* p, uint32_t bits) {
  const uint64_t a = ld64u(p) * 0x9E3779B97F4A7C15ull, b = ld64u(p + 8) * 0xC2B2AE3D27D4EB4Full;
  return (uint32_t)(((a ^ ((b << 31) | (b >> 33))) * 0x165667B19E3779F9ull) >> (64 - bits));
}

__device__ __forceinline__ uint32_t hash4(const uint8_t* p) { return (ld32u(p) * 2654435761u) >> (32 - kHashBits4); }

// Common prefix of a and b (a precedes b), at most limit bytes.
__device__ __forceinline__ uint32_t common(const uint8_t* a, const uint8_t* b, uint32_t limit) {
  uint32_t l = 0;
  while (l + 8 <= limit) {
    const uint64_t x = ld64u(a + l) ^ ld64u(b + l);
    if (x) return l + (__ffsll((long long)x) - 1) / 8;
    l += 8;
  }
  while (l < limit && a[l] == b[l]) l++;
  return l;
}

struct EncArgs {
  const uint8_t* in;
  uint64_t n, nb;
  uint32_t log2B, min_match, max_chain, w, adaptive, bits;
  unsigned long long* table;  // 2^bits: the earliest stride position with each key hash
  uint32_t* level;            // per block
  // the blocks of the current launch: [c0, c1), window start ws (blocks
  // below it, all of level below 3, may be sources)
  uint64_t c0, c1, ws;
  uint16_t* prev;     // per position of the chunk: distance to the previous one with the same 4-byte hash (0: none)
  uint16_t* lens;     // per position: in-block candidate length (low byte), external (high byte), capped at kCap
  uint64_t* q_in;     // per position: the in-block candidate's source
  uint64_t* q_ex;     // per position: the external candidate's source
  uint8_t* wave;      // per position: resolution wave of the byte (0: literal)
  uint32_t* tok;      // per chunk block: tok_cap x (lit_run, match_len, src lo, src hi)
  uint32_t tok_cap;
  uint32_t* ntok;     // per chunk block
  uint32_t* status;   // first error
  unsigned long long* stats;  // n_tokens, n_matches, literal, match, match_src bytes
};

// ---------------------------------------------------------------- the table

// Every stride position's 16-byte key: the table keeps the earliest.
__global__ void table_kernel(EncArgs a) {
  const uint64_t nkeys = a.n >= kKey ? (a.n - kKey) / kStride + 1 : 0;
  for (uint64_t k = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; k < nkeys; k += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t q = k * kStride;
    atomicMin(a.table + hash_key(a.in + q, a.bits), (unsigned long long)q);
  }
}

// ------------------------------------------------------- in-block chains

// A warp per block: positions in order, 32 at a time; a position's link is
// the nearest earlier one of the block with the same 4-byte hash (found
// among the lanes with __match_any_sync, else in the warp's bucket heads).
__global__ void chain_kernel(EncArgs a) {
  extern __shared__ uint32_t heads[];  // [warps][4096]
  const uint32_t lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  uint32_t* head = heads + (wid << kHashBits4);
  const uint64_t b = a.c0 + blockIdx.x * (blockDim.x >> 5) + wid;
  if (b >= a.c1) return;
  for (uint32_t i = lane; i < (1u << kHashBits4); i += 32) head[i] = 0xffffffffu;
  __syncwarp();
  const uint64_t B = 1ull << a.log2B, bstart = b << a.log2B, base = a.c0 << a.log2B;
  const uint32_t blen = (uint32_t)min(B, a.n - bstart);
  for (uint32_t c = 0; c < blen; c += 32) {
    const uint32_t p = c + lane;
    const bool valid = p + 4 <= blen;
    const uint32_t h = valid ? hash4(a.in + bstart + p) : (1u << kHashBits4) + lane;  // invalid lanes alone
    const uint32_t grp = __match_any_sync(kFull, h);
    const uint32_t below = grp & lanemask_lt();
    uint32_t pp = 0xffffffffu;
    if (valid) pp = below ? c + (31 - __clz(below)) : head[h];
    __syncwarp();
    if (valid && !(grp >> lane >> 1)) head[h] = p;  // the group's last lane is the new head
    __syncwarp();
    if (p < blen) a.prev[bstart - base + p] = (valid && pp != 0xffffffffu) ? (uint16_t)(p - pp) : (uint16_t)0;
  }
}

// ------------------------------------------------------ candidate search

// Bytes from q a match of block b may read without entering a block it may
// not read (its own block, or blocks below the window start of level below
// 3), at most want.
__device__ __forceinline__ uint32_t span(const EncArgs& a, uint64_t q, uint64_t b, uint32_t want) {
  uint64_t k = q >> a.log2B;
  uint32_t got = 0;
  while (got < want) {
    if (k != b && (k >= a.ws || a.level[k] >= 3)) break;
    const uint64_t end = (k + 1) << a.log2B;
    got = (uint32_t)min((uint64_t)want, end - q);
    k++;
  }
  return got;
}

// A thread per position of the launch's blocks: the best in-block candidate
// (its chain, most recent first, max_chain deep) and the best external one
// (earliest occurrences of the keys at p .. p + 7, shifted back), each the
// longest measured up to kCap bytes (ties: the smaller source).
__global__ void candidate_kernel(EncArgs a) {
  const uint64_t base = a.c0 << a.log2B, end = min(a.n, a.c1 << a.log2B);
  for (uint64_t p = base + blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; p < end;
       p += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t b = p >> a.log2B, bstart = b << a.log2B;
    const uint64_t bend = min((uint64_t)a.n, (uint64_t)(bstart + (1ull << a.log2B)));
    const uint32_t room = (uint32_t)(bend - p), lim = min(room, kCap);
    uint32_t li = 0, le = 0;
    uint64_t qi = 0, qe = 0;
    if (room >= a.min_match) {
      uint32_t d = a.prev[p - base];
      uint64_t q = p;
      for (uint32_t depth = 0; d && depth < a.max_chain; depth++) {
        if (d > q - bstart) break;  // links stay inside the block
        q -= d;
        const uint32_t l = common(a.in + q, a.in + p, lim);
        if (l > li) {
          li = l;
          qi = q;
        }
        d = a.prev[q - base];
      }
      for (uint32_t j = 0; j < kStride; j++) {
        const uint64_t x = p + j;
        if (x + kKey > a.n) break;
        const unsigned long long qq = a.table[hash_key(a.in + x, a.bits)];
        if (qq == kEmpty || qq < j) continue;
        q = qq - j;
        if (q >= p) continue;
        uint32_t l = common(a.in + q, a.in + p, lim);
        if (q >= bstart) {  // an earlier occurrence inside the block
          if (l > li || (l == li && q < qi)) {
            li = l;
            qi = q;
          }
          continue;
        }
        l = span(a, q, b, l);
        if (l > le || (l == le && q < qe)) {
          le = l;
          qe = q;
        }
      }
    }
    if (li < a.min_match) li = 0;
    if (le < a.min_match) le = 0;
    a.lens[p - base] = (uint16_t)(li | (le << 8));
    a.q_in[p - base] = qi;
    a.q_ex[p - base] = qe;
  }
}

// ----------------------------------------------------------- greedy parse

// The resolution wave a match from q of len bytes at p would take: 1 + the
// deepest wave among the bytes of its own block it reads (literals and
// bytes of earlier blocks are wave 0).
__device__ __forceinline__ uint32_t wave_of(const uint8_t* wv, uint64_t bstart, uint64_t q, uint64_t len,
                                            uint64_t p) {
  const uint64_t lo = max(q, bstart), hi = min(q + len, p);
  uint32_t w = 0;
  for (uint64_t k = lo; k < hi && w < kMaxWave; k++) w = max(w, (uint32_t)wv[k - bstart]);
  return w + 1;
}

// A thread per block: the greedy walk over its positions.  At each, both
// candidates are extended past the measured cap, a candidate deeper than
// kMaxWave is refused, and of the rest the longer one is taken -- except
// that a shallower one within max(4, len / 8) bytes of the longer wins.
__global__ void parse_kernel(EncArgs a) {
  const uint64_t b = a.c0 + blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (b >= a.c1) return;
  const uint64_t base = a.c0 << a.log2B, bstart = b << a.log2B;
  const uint64_t bend = min((uint64_t)a.n, (uint64_t)(bstart + (1ull << a.log2B)));
  uint8_t* wv = a.wave + (bstart - base);
  uint32_t* tk = a.tok + (b - a.c0) * (uint64_t)a.tok_cap * 4;
  uint32_t nt = 0, lit = 0;
  unsigned long long n_match = 0, mbytes = 0, msrc = 0, lbytes = 0;
  uint64_t p = bstart;
  while (p < bend) {
    // eight positions without a candidate at once (16-byte loads of the
    // candidate lengths; the wave bytes of eight literals as one word)
    if (((p - base) & 7) == 0 && p + 8 <= bend) {
      const uint4 v = *reinterpret_cast<const uint4*>(a.lens + (p - base));
      if ((v.x | v.y | v.z | v.w) == 0) {
        *reinterpret_cast<uint64_t*>(wv + (p - bstart)) = 0;
        lit += 8;
        lbytes += 8;
        p += 8;
        continue;
      }
    }
    const uint32_t ll = a.lens[p - base];
    uint32_t best_len = 0, best_w = 0;
    uint64_t best_q = 0;
    if (ll) {
      const uint32_t room = (uint32_t)(bend - p);
      auto consider = [&](uint64_t q, uint32_t l) {
        if (l < a.min_match) return;
        const uint32_t w = wave_of(wv, bstart, q, l, p);
        if (w > kMaxWave) return;
        const uint32_t slack = max(4u, max(l, best_len) / 8);
        bool take;
        if (!best_len) take = true;
        else if (w < best_w) take = l + slack >= best_len;
        else if (w > best_w) take = l > best_len + max(4u, l / 8);
        else take = l > best_len || (l == best_len && q < best_q);
        if (take) {
          best_len = l;
          best_q = q;
          best_w = w;
        }
      };
      const uint32_t li = ll & 0xff, le = ll >> 8;
      if (li) {
        const uint64_t q = a.q_in[p - base];
        uint32_t l = li;
        if (li == kCap && room > kCap) l = kCap + common(a.in + q + kCap, a.in + p + kCap, room - kCap);
        consider(q, l);
      }
      if (le) {
        const uint64_t q = a.q_ex[p - base];
        uint32_t l = le;
        if (le == kCap && room > kCap) l = span(a, q, b, kCap + common(a.in + q + kCap, a.in + p + kCap, room - kCap));
        consider(q, l);
      }
    }
    if (best_len >= a.min_match && nt + 1 < a.tok_cap) {
      uint32_t* t = tk + 4 * nt++;
      t[0] = lit;
      t[1] = best_len;
      t[2] = (uint32_t)best_q;
      t[3] = (uint32_t)(best_q >> 32);
      for (uint64_t k = p; k < p + best_len; k++) wv[k - bstart] = (uint8_t)best_w;
      n_match++;
      mbytes += best_len;
      msrc += min((uint64_t)best_len, p - best_q);
      lit = 0;
      p += best_len;
    } else {
      wv[p - bstart] = 0;
      lit++;
      lbytes++;
      p++;
    }
  }
  uint32_t* t = tk + 4 * nt++;  // the last token: literals only
  t[0] = lit;
  t[1] = 0;
  t[2] = t[3] = 0;
  a.ntok[b - a.c0] = nt;
  atomicAdd(a.stats + 0, (unsigned long long)nt);
  atomicAdd(a.stats + 1, n_match);
  atomicAdd(a.stats + 2, lbytes);
  atomicAdd(a.stats + 3, mbytes);
  atomicAdd(a.stats + 4, msrc);
}

// ------------------------------------------------------------ block coder

struct CodeArgs {
  EncArgs e;
  uint8_t* syms;       // per chunk block: sym_cap bytes, the three streams' symbols one after another
  uint32_t sym_cap;
  uint32_t* tmp;       // per chunk block: one word per symbol of the longest stream (pushes of the encode)
  uint32_t tmp_cap;
  uint8_t* pay;        // per chunk block: pay_cap bytes, the block's payload
  uint32_t pay_cap;
  ace_block_dir* dir;  // per block of the archive (stream offsets relative to the block's payload for now)
  uint32_t* pay_bytes; // per chunk block
  uint32_t* iv;        // per block of the archive: up to kHead / 2 (first, last) pairs
  uint32_t* n_iv;      // per block of the archive
};

constexpr uint32_t kIvCap = kHead / 2;  // runs of set bits in a kHead-bit map

// Frequencies of a stream as the host encoder quantises them: f_s =
// max(1, floor(n_s 4096 / n)); a shortfall goes to the most frequent symbol
// (lowest on ties), an excess is taken one at a time from the largest
// frequency above 1 (lowest on ties).  cnt: the histogram in shared memory;
// leaves f | c << 16 per symbol in fc.  Lane l holds symbols 8l .. 8l + 7.
__device__ void quantise_warp(const uint32_t* cnt, uint32_t n, uint32_t* fc, uint32_t lane) {
  uint32_t f[8], sum = 0, best = 0, most = 0;
#pragma unroll
  for (int j = 0; j < 8; j++) {
    const uint32_t s = 8 * lane + j, c = cnt[s];
    f[j] = c ? max(1u, (uint32_t)(((uint64_t)c * ACE_SCALE) / n)) : 0u;
    sum += f[j];
    if (c > best) {
      best = c;
      most = s;
    }
  }
  // most frequent, lowest symbol on ties: (count, -symbol) maximal
#pragma unroll
  for (int d = 16; d; d >>= 1) {
    const uint32_t ob = __shfl_xor_sync(kFull, best, d), om = __shfl_xor_sync(kFull, most, d);
    if (ob > best || (ob == best && om < most)) {
      best = ob;
      most = om;
    }
  }
#pragma unroll
  for (int d = 16; d; d >>= 1) sum += __shfl_xor_sync(kFull, sum, d);
  if (sum < ACE_SCALE && (most >> 3) == lane) {
#pragma unroll
    for (int j = 0; j < 8; j++)
      if (8 * lane + j == most) f[j] += ACE_SCALE - sum;
  }
  while (sum > ACE_SCALE) {  // warp-uniform: sum is the same on every lane
    uint32_t bf = 0, bs = 0xffffffffu;
#pragma unroll
    for (int j = 0; j < 8; j++)
      if (f[j] > 1 && f[j] > bf) {
        bf = f[j];
        bs = 8 * lane + j;
      }
#pragma unroll
    for (int d = 16; d; d >>= 1) {
      const uint32_t of = __shfl_xor_sync(kFull, bf, d), os = __shfl_xor_sync(kFull, bs, d);
      if (of > bf || (of == bf && os < bs)) {
        bf = of;
        bs = os;
      }
    }
    if ((bs >> 3) == lane) {
#pragma unroll
      for (int j = 0; j < 8; j++)
        if (8 * lane + j == bs) f[j]--;
    }
    sum--;
  }
  uint32_t tot = 0;
#pragma unroll
  for (int j = 0; j < 8; j++) tot += f[j];
  uint32_t c = warp_incl_sum(tot, lane) - tot;
#pragma unroll
  for (int j = 0; j < 8; j++) {
    fc[8 * lane + j] = f[j] | (c << 16);
    c += f[j];
  }
  __syncwarp();
}

// One stream of n symbols into out (16-byte aligned): its rANS payload
// (32 final states, present bitmap, frequencies, renormalisation bytes), or,
// with adaptive set and rANS not shrinking it, the symbols themselves.
// The encode walks the symbols from the last to the first, symbol i on state
// i mod 32, pushing a state's low byte while x >= 2^19 f_s, then x <-
// (x / f_s) 4096 + x mod f_s + c_s; the pushes are then laid out in symbol
// order, each symbol's bytes last push first, which is the byte order the
// decoder reads.  Returns the stream's bytes; sets *mode.
__device__ uint32_t code_stream_warp(const uint8_t* sym, uint32_t n, uint8_t* out, uint32_t* tmp, uint32_t* cnt,
                                     uint32_t* fc, bool adaptive, uint32_t* mode, uint32_t lane) {
  *mode = 0;
  if (n == 0) return 0;
  for (uint32_t s = lane; s < 256; s += 32) cnt[s] = 0;
  __syncwarp();
  for (uint32_t i = lane; i < n; i += 32) atomicAdd(cnt + sym[i], 1u);
  __syncwarp();
  quantise_warp(cnt, n, fc, lane);
  // backward: pushes per symbol (count in bits 16..17, bytes below)
  uint32_t x = ACE_RANS_L, pushes = 0;
  const uint32_t rounds = (n + 31) / 32;
  for (uint32_t r = rounds; r-- > 0;) {
    const uint32_t i = 32 * r + lane;
    if (i < n) {
      const uint32_t e = fc[sym[i]], f = e & 0xffffu, c = e >> 16;
      const uint32_t lim = f << (ACE_SCALE_BITS + 7);  // (L / 4096) * 256 * f = 2^19 f
      uint32_t k = 0, bytes = 0;
      while (x >= lim) {
        bytes |= (x & 255u) << (8 * k);
        x >>= 8;
        k++;
      }
      x = ((x / f) << ACE_SCALE_BITS) + (x % f) + c;
      tmp[i] = bytes | (k << 16);
      pushes += k;
    }
  }
#pragma unroll
  for (int d = 16; d; d >>= 1) pushes += __shfl_xor_sync(kFull, pushes, d);
  // the present symbols: bitmap byte l holds symbols 8l .. 8l + 7
  uint32_t bm = 0;
#pragma unroll
  for (int j = 0; j < 8; j++) bm |= (fc[8 * lane + j] & 0xffffu) ? 1u << j : 0u;
  const uint32_t np = __popc(bm);
  const uint32_t first = warp_incl_sum(np, lane) - np;
  const uint32_t present = __shfl_sync(kFull, first + np, 31);
  const uint32_t head = ACE_STREAM_HEAD + ((2 * present + 15) & ~15u);
  if (adaptive && head + pushes >= n) {  // stored: the symbols verbatim
    for (uint32_t i = lane; i < n; i += 32) out[i] = sym[i];
    for (uint32_t i = n + lane; i < ((n + 15) & ~15u); i += 32) out[i] = 0;
    *mode = 1;
    return n;
  }
  reinterpret_cast<uint32_t*>(out)[lane] = x;  // the final states: the decoder's entry point
  out[128 + lane] = (uint8_t)bm;
  uint32_t k = first;
#pragma unroll
  for (int j = 0; j < 8; j++) {
    const uint32_t f = fc[8 * lane + j] & 0xffffu;
    if (f) {
      out[ACE_STREAM_HEAD + 2 * k] = (uint8_t)f;
      out[ACE_STREAM_HEAD + 2 * k + 1] = (uint8_t)(f >> 8);
      k++;
    }
  }
  for (uint32_t i = ACE_STREAM_HEAD + 2 * present + lane; i < head; i += 32) out[i] = 0;
  // forward: each symbol's bytes at the running count of the pushes before it
  uint32_t run = 0;
  for (uint32_t r = 0; r < rounds; r++) {
    const uint32_t i = 32 * r + lane;
    const uint32_t t = i < n ? tmp[i] : 0u, kk = t >> 16;
    const uint32_t incl = warp_incl_sum(kk, lane), at = head + run + incl - kk;
    if (kk == 2) {
      out[at] = (uint8_t)(t >> 8);
      out[at + 1] = (uint8_t)t;
    } else if (kk == 1) {
      out[at] = (uint8_t)t;
    }
    run += __shfl_sync(kFull, incl, 31);
  }
  const uint32_t total = head + pushes;
  for (uint32_t i = total + lane; i < ((total + 15) & ~15u); i += 32) out[i] = 0;
  __syncwarp();
  return total;
}

// A warp per block: the token streams (literals in output order; lengths:
// the escape values, then two codes per token; offsets: each match's
// absolute source, w bytes), each coded, one after another 16-byte aligned
// in the block's payload; the directory entry; the dependency runs (a bit
// per earlier block a match reads, all below the window start) and the
// block's level.
__global__ void code_kernel(CodeArgs ca) {
  __shared__ uint32_t s_cnt[8][256], s_fc[8][256], s_bits[8][kHead / 32 + 1], s_misc[8][4];
  const EncArgs& a = ca.e;
  const uint32_t lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const uint64_t b = a.c0 + blockIdx.x * (blockDim.x >> 5) + wid;
  if (b >= a.c1) return;
  const uint64_t cb = b - a.c0, bstart = b << a.log2B;
  const uint32_t* tk = a.tok + cb * (uint64_t)a.tok_cap * 4;
  const uint32_t nt = a.ntok[cb], nm = nt - 1, w = a.w;
  uint8_t* lit = ca.syms + cb * (uint64_t)ca.sym_cap;
  // token positions: run starts and literal positions (exclusive scans)
  uint32_t dst = 0, lpos = 0, nesc = 0;
  for (uint32_t i = lane; i < kHead / 32 + 1; i += 32) s_bits[wid][i] = 0;
  __syncwarp();
  uint32_t* lens_base = nullptr;
  // pass 1: escape counts and literal total
  uint32_t esc_total = 0, lit_total = 0;
  for (uint32_t t0 = 0; t0 < nt; t0 += 32) {
    const uint32_t t = t0 + lane;
    uint32_t e = 0, lr = 0;
    if (t < nt) {
      lr = tk[4 * t];
      e = (lr >= 255) + (tk[4 * t + 1] >= 255);
    }
#pragma unroll
    for (int d = 16; d; d >>= 1) {
      e += __shfl_xor_sync(kFull, e, d);
      lr += __shfl_xor_sync(kFull, lr, d);
    }
    esc_total += e;
    lit_total += lr;
  }
  uint8_t* lenp = lit + lit_total;              // lengths stream: 2 esc_total + 2 nt bytes
  uint8_t* offp = lenp + 2 * esc_total + 2 * nt;  // offsets stream: w nm bytes
  (void)lens_base;
  // pass 2: the three streams' symbols, and the dependency bits
  const uint64_t B = 1ull << a.log2B;
  for (uint32_t t0 = 0; t0 < nt; t0 += 32) {
    const uint32_t t = t0 + lane;
    uint32_t lr = 0, ml = 0;
    uint64_t src = 0;
    if (t < nt) {
      lr = tk[4 * t];
      ml = tk[4 * t + 1];
      src = (uint64_t)tk[4 * t + 2] | ((uint64_t)tk[4 * t + 3] << 32);
    }
    const uint32_t run = lr + ml, e = (t < nt) ? (lr >= 255) + (ml >= 255) : 0u;
    const uint32_t ri = warp_incl_sum(run, lane), li = warp_incl_sum(lr, lane), ei = warp_incl_sum(e, lane);
    const uint32_t my_dst = dst + ri - run, my_lit = lpos + li - lr, my_esc = nesc + ei - e;
    if (t < nt) {
      for (uint32_t k = 0; k < lr; k++) lit[my_lit + k] = a.in[bstart + my_dst + k];
      uint32_t ec = my_esc;
      const uint32_t v[2] = {lr, ml};
      for (int q = 0; q < 2; q++) {
        if (v[q] < 255) {
          lenp[2 * esc_total + 2 * t + q] = (uint8_t)v[q];
        } else {
          lenp[2 * esc_total + 2 * t + q] = 255;
          lenp[2 * ec] = (uint8_t)(v[q] - 255);
          lenp[2 * ec + 1] = (uint8_t)((v[q] - 255) >> 8);
          ec++;
        }
      }
      if (t < nm) {
        for (uint32_t k = 0; k < w; k++) offp[w * t + k] = (uint8_t)(src >> (8 * k));
        const uint64_t D = bstart + my_dst + lr;
        if (ml && src < bstart) {  // blocks before this one that the match reads
          const uint64_t rl = min((uint64_t)ml, D - src);
          const uint64_t k0 = src >> a.log2B, k1 = min((src + rl - 1) >> a.log2B, b - 1);
          for (uint64_t k = k0; k <= k1 && k < kHead; k++) atomicOr(&s_bits[wid][k >> 5], 1u << (k & 31));
        }
      }
    }
    dst += __shfl_sync(kFull, ri, 31);
    lpos += __shfl_sync(kFull, li, 31);
    nesc += __shfl_sync(kFull, ei, 31);
  }
  __syncwarp();
  // the three streams
  uint8_t* pay = ca.pay + cb * (uint64_t)ca.pay_cap;
  uint32_t* tmp = ca.tmp + cb * (uint64_t)ca.tmp_cap;
  const uint8_t* streams[3] = {lit, lenp, offp};
  const uint32_t ns[3] = {lit_total, 2 * esc_total + 2 * nt, w * nm};
  ace_block_dir d;
  memset(&d, 0, sizeof d);
  uint32_t off = 0;
  for (int k = 0; k < 3; k++) {
    uint32_t mode;
    const uint32_t bytes = code_stream_warp(streams[k], ns[k], pay + off, tmp, s_cnt[wid], s_fc[wid], a.adaptive != 0,
                                            &mode, lane);
    d.stream_off[k] = off;
    d.stream_bytes[k] = bytes;
    d.nsym[k] = ns[k];
    d.mode[k] = (uint8_t)mode;
    off += (bytes + 15) & ~15u;
  }
  d.ntok = nt;
  d.nesc = esc_total;
  // dependency runs and the level: 1 + the deepest block read
  uint32_t lv = 0;
  for (uint32_t k = lane; k < kHead && k < b; k += 32)
    if (s_bits[wid][k >> 5] >> (k & 31) & 1) lv = max(lv, a.level[k] + 1);
#pragma unroll
  for (int dd = 16; dd; dd >>= 1) lv = max(lv, __shfl_xor_sync(kFull, lv, dd));
  if (lane == 0) {
    uint32_t cnt = 0, k = 0;
    uint32_t* iv = ca.iv + b * (uint64_t)(2 * kIvCap);
    const uint32_t top = (uint32_t)min((uint64_t)b, (uint64_t)kHead);
    while (k < top) {
      if (!(s_bits[wid][k >> 5] >> (k & 31) & 1)) {
        k++;
        continue;
      }
      uint32_t e = k;
      while (e + 1 < top && (s_bits[wid][(e + 1) >> 5] >> ((e + 1) & 31) & 1)) e++;
      iv[2 * cnt] = k;
      iv[2 * cnt + 1] = e;
      cnt++;
      k = e + 1;
    }
    ca.n_iv[b] = cnt;
    a.level[b] = lv;
    ca.dir[b] = d;
    ca.pay_bytes[cb] = off;
  }
  (void)B;
}

// ------------------------------------------------------ payload placement

struct EncHdr {
  uint32_t status;
  uint32_t max_level;
  uint64_t payload;   // payload bytes placed so far
  uint64_t n_iv;      // dependency runs in the archive
  unsigned long long stats[5];
  uint8_t pad[256 - 64];
};
static_assert(sizeof(EncHdr) == 256, "encoder header");

struct PlaceArgs {
  EncHdr* h;
  const uint32_t* pay_bytes;  // per chunk block
  uint64_t* pay_off;          // per chunk block: offset from the payload's start
  ace_block_dir* dir;
  uint64_t c0, cn;            // the chunk's first block and block count
  const uint8_t* pay;
  uint32_t pay_cap;
  uint8_t* dst;               // where the payload is assembled (the archive buffer's tail)
  uint64_t dst_cap;           // bytes available there
};

// One CTA: the chunk's block payloads laid end to end after the payload so
// far (each a multiple of 16 bytes), their directory offsets made relative
// to the payload's start.
__global__ void place_scan_kernel(PlaceArgs p) {
  __shared__ unsigned long long carry, wsum[32];
  const uint32_t lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (threadIdx.x == 0) carry = p.h->payload;
  __syncthreads();
  for (uint64_t c0 = 0; c0 < p.cn; c0 += blockDim.x) {
    const uint64_t i = c0 + threadIdx.x;
    const unsigned long long v = i < p.cn ? p.pay_bytes[i] : 0;
    unsigned long long incl = v;
    for (int d = 1; d < 32; d <<= 1) {
      const unsigned long long u = __shfl_up_sync(kFull, incl, d);
      if (lane >= (uint32_t)d) incl += u;
    }
    if (lane == 31) wsum[wid] = incl;
    __syncthreads();
    if (wid == 0) {
      unsigned long long x = lane < nw ? wsum[lane] : 0, xi = x;
      for (int d = 1; d < 32; d <<= 1) {
        const unsigned long long u = __shfl_up_sync(kFull, xi, d);
        if (lane >= (uint32_t)d) xi += u;
      }
      if (lane < nw) wsum[lane] = xi - x;
    }
    __syncthreads();
    const unsigned long long at = carry + wsum[wid] + incl - v;
    if (i < p.cn) {
      p.pay_off[i] = at;
      ace_block_dir& d = p.dir[p.c0 + i];
      for (int k = 0; k < 3; k++) d.stream_off[k] += at;
    }
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) carry = at + v;
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    if (carry > p.dst_cap) record_error(&p.h->status, &p.h->status, &p.h->status, ACE_E_NOMEM, 0, 0);
    p.h->payload = carry;
  }
}

// A warp per block: its payload to its place (16-byte pieces).
__global__ void place_copy_kernel(PlaceArgs p) {
  const uint32_t lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const uint64_t i = blockIdx.x * (uint64_t)(blockDim.x >> 5) + wid;
  if (i >= p.cn || *(volatile uint32_t*)&p.h->status) return;
  const uint4* src = reinterpret_cast<const uint4*>(p.pay + i * (uint64_t)p.pay_cap);
  uint4* dst = reinterpret_cast<uint4*>(p.dst + p.pay_off[i]);
  const uint32_t n16 = p.pay_bytes[i] / 16;
  for (uint32_t k = lane; k < n16; k += 32) dst[k] = src[k];
}

// ---------------------------------------------------------------- assembly

struct AsmArgs {
  EncHdr* h;
  const uint32_t* n_iv;   // per block
  const uint32_t* iv;     // per block: kIvCap pairs
  uint32_t* dep_ptr;      // scratch: nb + 1
  const uint32_t* level;
  uint64_t nb;
};

// One CTA: the dependency table's pointers (exclusive prefix of the runs),
// the total, and the deepest level.
__global__ void deps_scan_kernel(AsmArgs a) {
  __shared__ uint32_t carry, wsum[32], lmax;
  const uint32_t lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (threadIdx.x == 0) {
    carry = 0;
    lmax = 0;
  }
  __syncthreads();
  for (uint64_t c0 = 0; c0 < a.nb; c0 += blockDim.x) {
    const uint64_t i = c0 + threadIdx.x;
    const uint32_t v = i < a.nb ? a.n_iv[i] : 0;
    if (i < a.nb) atomicMax(&lmax, a.level[i]);
    const uint32_t incl = warp_incl_sum(v, lane);
    if (lane == 31) wsum[wid] = incl;
    __syncthreads();
    if (wid == 0) {
      const uint32_t x = lane < nw ? wsum[lane] : 0, xi = warp_incl_sum(x, lane);
      if (lane < nw) wsum[lane] = xi - x;
    }
    __syncthreads();
    const uint32_t at = carry + wsum[wid] + incl - v;
    if (i < a.nb) a.dep_ptr[i] = at;
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) carry = at + v;
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    a.dep_ptr[a.nb] = carry;
    a.h->n_iv = carry;
    a.h->max_level = lmax;
  }
}

// The directory and the dependency table into the archive: pointers, then
// each block's runs at its pointer.
__global__ void deps_write_kernel(AsmArgs a, const ace_block_dir* dir, uint8_t* arc, uint64_t dir_off,
                                  uint64_t deps_off) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i <= a.nb; i += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t* ptr = reinterpret_cast<uint32_t*>(arc + deps_off);
    ptr[i] = a.dep_ptr[i];
    if (i == a.nb) continue;
    reinterpret_cast<ace_block_dir*>(arc + dir_off)[i] = dir[i];
    uint32_t* ivs = ptr + a.nb + 1 + 2ull * a.dep_ptr[i];
    const uint32_t* src = a.iv + i * (uint64_t)(2 * kIvCap);
    for (uint32_t k = 0; k < 2 * a.n_iv[i]; k++) ivs[k] = src[k];
  }
}

}  // namespace

// --------------------------------------------------------------- host side

namespace {

struct EncLayout {
  uint64_t table, level, dir, iv, n_iv, dep_ptr, hdr, prev, lens, q_in, q_ex, wave, tok, ntok, syms, tmp, pay,
      pay_bytes, pay_off, total;
  uint64_t nb, chunk, reserve, arc_bound;
  uint32_t bits, tok_cap, sym_cap, tmp_cap, pay_cap;
};

inline uint64_t a256(uint64_t v) { return (v + 255) & ~255ull; }

ace_status enc_layout(uint64_t n, const ace_encode_params* p, EncLayout* L) {
  if (!p || p->log2_block < ACE_MIN_LOG2_BLOCK || p->log2_block > ACE_MAX_LOG2_BLOCK || p->min_match < 4 ||
      p->adaptive > 1 || p->max_chain > kMaxChain)
    return ACE_E_INVAL;
  if (p->off_width != 0 && p->off_width != 4 && p->off_width != 5) return ACE_E_INVAL;
  if (p->off_width == 4 && n > (1ull << 32)) return ACE_E_INVAL;
  const uint64_t B = 1ull << p->log2_block;
  L->nb = (n + B - 1) / B;
  if (L->nb > 0xFFFFFFF0ull) return ACE_E_INVAL;
  uint64_t want = std::max<uint64_t>(1, n / kStride);
  L->bits = 10;
  while (L->bits < 27 && (1ull << L->bits) < want) L->bits++;
  const uint64_t chunk = p->threads ? p->threads : std::max<uint64_t>(kWin, (64ull << 20) >> p->log2_block);
  L->chunk = std::max<uint64_t>(1, std::min<uint64_t>(chunk, std::max<uint64_t>(L->nb, 1)));
  L->tok_cap = (uint32_t)(B / p->min_match + 2);
  L->sym_cap = (uint32_t)align16(B + 11ull * L->tok_cap);
  L->tmp_cap = L->sym_cap;
  L->pay_cap = (uint32_t)align16(3ull * (ACE_STREAM_HEAD + 2 * 256 + 16) + 2ull * L->sym_cap + 64);
  const uint64_t nb = L->nb, C = L->chunk, cb = C * B;
  uint64_t o = 0;
  L->hdr = o;
  o = a256(o + sizeof(EncHdr));
  L->table = o;
  o = a256(o + (8ull << L->bits));
  L->level = o;
  o = a256(o + 4 * nb);
  L->dir = o;
  o = a256(o + 64 * nb);
  L->iv = o;
  o = a256(o + 8ull * kIvCap * nb);
  L->n_iv = o;
  o = a256(o + 4 * nb);
  L->dep_ptr = o;
  o = a256(o + 4 * (nb + 1));
  L->prev = o;
  o = a256(o + 2 * cb);
  L->lens = o;
  o = a256(o + 2 * cb);
  L->q_in = o;
  o = a256(o + 8 * cb);
  L->q_ex = o;
  o = a256(o + 8 * cb);
  L->wave = o;
  o = a256(o + cb);
  L->tok = o;
  o = a256(o + 16ull * L->tok_cap * C);
  L->ntok = o;
  o = a256(o + 4 * C);
  L->syms = o;
  o = a256(o + (uint64_t)L->sym_cap * C);
  L->tmp = o;
  o = a256(o + 4ull * L->tmp_cap * C);
  L->pay = o;
  o = a256(o + (uint64_t)L->pay_cap * C);
  L->pay_bytes = o;
  o = a256(o + 4 * C);
  L->pay_off = o;
  o = a256(o + 8 * C);
  L->total = o;
  // the payload is assembled after room for the largest header, directory
  // and dependency table, then moved down against the table's real size
  L->reserve = a256(sizeof(ace_file_header) + 64 * nb + 4 * (nb + 1) + 8ull * kIvCap * nb);
  L->arc_bound = L->reserve + nb * (uint64_t)L->pay_cap + 256;
  return ACE_OK;
}

}  // namespace

extern "C" {

ace_status ace_encode_gpu_size(uint64_t n, const ace_encode_params* params, uint64_t* scratch_bytes,
                               uint64_t* arc_bound) {
  EncLayout L;
  ace_status rc = enc_layout(n, params, &L);
  if (rc) return rc;
  if (scratch_bytes) *scratch_bytes = L.total;
  if (arc_bound) *arc_bound = L.arc_bound;
  return ACE_OK;
}

#define ENC_TRY(x)                              \
  do {                                          \
    if ((x) != cudaSuccess) return ACE_E_CUDA;  \
  } while (0)

ace_status ace_encode_gpu(const void* d_in, uint64_t n, const ace_encode_params* params, void* d_scratch,
                          uint64_t scratch_bytes, void* d_arc, uint64_t arc_cap, uint64_t* h_arc_len,
                          ace_encode_stats* h_stats, cudaStream_t s) {
  EncLayout L;
  ace_status rc = enc_layout(n, params, &L);
  if (rc) return rc;
  if ((!d_in && n) || !d_scratch || !d_arc || !h_arc_len) return ACE_E_INVAL;
  if ((reinterpret_cast<uintptr_t>(d_scratch) & 255) || (reinterpret_cast<uintptr_t>(d_arc) & 255))
    return ACE_E_INVAL;
  if (scratch_bytes < L.total || arc_cap < L.reserve + 256) return ACE_E_NOMEM;
  uint8_t* base = static_cast<uint8_t*>(d_scratch);
  uint8_t* arc = static_cast<uint8_t*>(d_arc);
  const uint64_t nb = L.nb, B = 1ull << params->log2_block;
  const uint32_t w = (n > (1ull << 32) || params->off_width == 5) ? 5 : 4;
  EncHdr* hdr = reinterpret_cast<EncHdr*>(base + L.hdr);
  ENC_TRY(cudaMemsetAsync(base + L.hdr, 0, sizeof(EncHdr), s));
  ENC_TRY(cudaMemsetAsync(base + L.table, 0xff, 8ull << L.bits, s));
  if (nb) ENC_TRY(cudaMemsetAsync(base + L.level, 0, 4 * nb, s));
  EncArgs e{};
  e.in = static_cast<const uint8_t*>(d_in);
  e.n = n;
  e.nb = nb;
  e.log2B = params->log2_block;
  e.min_match = params->min_match;
  e.max_chain = params->max_chain ? params->max_chain : 16;
  e.w = w;
  e.adaptive = params->adaptive;
  e.bits = L.bits;
  e.table = reinterpret_cast<unsigned long long*>(base + L.table);
  e.level = reinterpret_cast<uint32_t*>(base + L.level);
  e.prev = reinterpret_cast<uint16_t*>(base + L.prev);
  e.lens = reinterpret_cast<uint16_t*>(base + L.lens);
  e.q_in = reinterpret_cast<uint64_t*>(base + L.q_in);
  e.q_ex = reinterpret_cast<uint64_t*>(base + L.q_ex);
  e.wave = base + L.wave;
  e.tok = reinterpret_cast<uint32_t*>(base + L.tok);
  e.tok_cap = L.tok_cap;
  e.ntok = reinterpret_cast<uint32_t*>(base + L.ntok);
  e.status = &hdr->status;
  e.stats = hdr->stats;
  CodeArgs ca;
  ca.syms = base + L.syms;
  ca.sym_cap = L.sym_cap;
  ca.tmp = reinterpret_cast<uint32_t*>(base + L.tmp);
  ca.tmp_cap = L.tmp_cap;
  ca.pay = base + L.pay;
  ca.pay_cap = L.pay_cap;
  ca.dir = reinterpret_cast<ace_block_dir*>(base + L.dir);
  ca.pay_bytes = reinterpret_cast<uint32_t*>(base + L.pay_bytes);
  ca.iv = reinterpret_cast<uint32_t*>(base + L.iv);
  ca.n_iv = reinterpret_cast<uint32_t*>(base + L.n_iv);
  PlaceArgs pa;
  pa.h = hdr;
  pa.pay_bytes = ca.pay_bytes;
  pa.pay_off = reinterpret_cast<uint64_t*>(base + L.pay_off);
  pa.dir = ca.dir;
  pa.pay = ca.pay;
  pa.pay_cap = L.pay_cap;
  pa.dst = arc + L.reserve;
  pa.dst_cap = arc_cap - L.reserve;
  if (n >= kKey) {
    const uint64_t nkeys = (n - kKey) / kStride + 1;
    table_kernel<<<(uint32_t)std::min<uint64_t>((nkeys + 255) / 256, 65535ull * 8), 256, 0, s>>>(e);
  }
  // launches: the first three windows one after another (a window takes
  // sources only from the windows before it), then every later block
  // taking sources only from the first three windows
  struct Piece {
    uint64_t c0, c1, ws;
  };
  std::vector<Piece> pieces;
  const uint64_t head = std::min<uint64_t>(nb, kHead);
  for (uint64_t w0 = 0; w0 < head; w0 += kWin)
    for (uint64_t c = w0; c < std::min(head, w0 + kWin); c += L.chunk)
      pieces.push_back({c, std::min({head, w0 + kWin, c + L.chunk}), w0});
  for (uint64_t c = head; c < nb; c += L.chunk) pieces.push_back({c, std::min(nb, c + L.chunk), head});
  constexpr uint32_t kChainWarps = 2;  // 16 KiB of bucket heads each: within the default shared memory
  for (const Piece& pc : pieces) {
    e.c0 = pc.c0;
    e.c1 = pc.c1;
    e.ws = pc.ws;
    const uint64_t cn = pc.c1 - pc.c0;
    chain_kernel<<<(uint32_t)((cn + kChainWarps - 1) / kChainWarps), 32 * kChainWarps,
                   kChainWarps * (4u << kHashBits4), s>>>(e);
    const uint64_t npos = std::min(n, pc.c1 * B) - pc.c0 * B;
    candidate_kernel<<<(uint32_t)std::min<uint64_t>((npos + 255) / 256, 152ull * 64), 256, 0, s>>>(e);
    parse_kernel<<<(uint32_t)((cn + 31) / 32), 32, 0, s>>>(e);
    ca.e = e;
    code_kernel<<<(uint32_t)((cn + 7) / 8), 256, 0, s>>>(ca);
    pa.c0 = pc.c0;
    pa.cn = cn;
    place_scan_kernel<<<1, 1024, 0, s>>>(pa);
    place_copy_kernel<<<(uint32_t)((cn + 7) / 8), 256, 0, s>>>(pa);
  }
  AsmArgs aa;
  aa.h = hdr;
  aa.n_iv = ca.n_iv;
  aa.iv = ca.iv;
  aa.dep_ptr = reinterpret_cast<uint32_t*>(base + L.dep_ptr);
  aa.level = e.level;
  aa.nb = nb;
  if (nb) deps_scan_kernel<<<1, 1024, 0, s>>>(aa);
  ENC_TRY(cudaGetLastError());
  EncHdr h;
  ENC_TRY(cudaMemcpyAsync(&h, hdr, sizeof h, cudaMemcpyDeviceToHost, s));
  ENC_TRY(cudaStreamSynchronize(s));
  if (h.status) return (ace_status)h.status;
  ace_file_header fh{};
  fh.magic = ACE_MAGIC;
  fh.version = ACE_VERSION;
  fh.n_streams = ACE_NSTREAMS;
  fh.n_states = ACE_NSTATES;
  fh.scale_bits = ACE_SCALE_BITS;
  fh.off_width = (uint8_t)w;
  fh.log2_block = (uint8_t)params->log2_block;
  fh.total_size = n;
  fh.n_blocks = nb;
  fh.dir_off = sizeof(ace_file_header);
  fh.deps_off = fh.dir_off + 64 * nb;
  fh.payload_off = align16(fh.deps_off + 4 * (nb + 1) + 8 * h.n_iv);
  fh.archive_bytes = align16(fh.payload_off + h.payload);
  if (fh.archive_bytes > arc_cap || fh.payload_off > L.reserve) return ACE_E_NOMEM;
  ENC_TRY(cudaMemsetAsync(arc, 0, fh.payload_off, s));
  if (nb) {
    deps_write_kernel<<<(uint32_t)std::min<uint64_t>((nb + 256) / 256, 65535), 256, 0, s>>>(aa, ca.dir, arc, fh.dir_off,
                                                                                           fh.deps_off);
    // the payload down to its place, in pieces no longer than the gap
    const uint64_t gap = L.reserve - fh.payload_off;
    for (uint64_t o = 0; o < h.payload;) {
      const uint64_t len = gap ? std::min(gap, h.payload - o) : h.payload;
      if (gap) ENC_TRY(cudaMemcpyAsync(arc + fh.payload_off + o, arc + L.reserve + o, len, cudaMemcpyDeviceToDevice, s));
      o += len;
    }
  }
  if (fh.archive_bytes > fh.payload_off + h.payload)
    ENC_TRY(cudaMemsetAsync(arc + fh.payload_off + h.payload, 0, fh.archive_bytes - fh.payload_off - h.payload, s));
  ENC_TRY(cudaMemcpyAsync(arc, &fh, sizeof fh, cudaMemcpyHostToDevice, s));
  ENC_TRY(cudaGetLastError());
  ENC_TRY(cudaStreamSynchronize(s));
  *h_arc_len = fh.archive_bytes;
  if (h_stats) {
    h_stats->n_tokens = h.stats[0];
    h_stats->n_matches = h.stats[1];
    h_stats->literal_bytes = h.stats[2];
    h_stats->match_bytes = h.stats[3];
    h_stats->match_src_bytes = h.stats[4];
    h_stats->n_dep_intervals = h.n_iv;
    h_stats->n_levels = nb ? h.max_level + 1 : 0;
    h_stats->reserved = 0;
  }
  return ACE_OK;
}

}  // extern "C"
