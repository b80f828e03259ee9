// Host encoder of the two-layer codec (CPU, multithreaded).
//
// Produces the archive layout of ace_format.h:
//  - match layer (Section 2): a greedy parse whose back-references are
//    absolute positions.  Candidates are (a) the earliest earlier occurrence
//    of any 16-byte key, found through a table built over the whole input
//    (the global match search), and (b) shorter repeats within the block,
//    found through a per-block hash chain.  Sources therefore sit either in
//    the block itself or at the earliest place a long string occurs, which
//    keeps block dependency levels shallow for the GPU decoder.  A match's
//    destination never crosses its block end.
//  - entropy layer (Section 3): each block's literal, length and offset
//    streams are rANS-coded on their own with 32 interleaved 32-bit states,
//    12-bit frequencies and byte renormalisation; the final states are stored
//    as the block's entry point.
//  - the dependency table: per block, the maximal runs of earlier blocks its
//    matches read (Section 2: a block decodes once those are present).
//
// Blocks are parsed and coded independently, so the archive is the same for
// any thread count.
#include <algorithm>
#include <atomic>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <new>
#include <thread>
#include <vector>

#include "ace.h"
#include "ace_format.h"

namespace {

constexpr int kKey = 16;        // long-key length for the global table
constexpr int kStride = 8;      // positions inserted into the global table
constexpr uint64_t kEmpty = ~0ull;
constexpr uint64_t kWindow = 64;   // blocks parsed together; they take no sources from each other
constexpr uint32_t kMaxLevel = 3;  // default cap on a block's dependency level
constexpr uint32_t kMaxWave = 3;   // cap on the in-block resolution wave of a match

inline uint64_t load64(const uint8_t* p) {
  uint64_t v;
  std::memcpy(&v, p, 8);
  return v;  // both supported hosts are little-endian
}

inline uint32_t load32(const uint8_t* p) {
  uint32_t v;
  std::memcpy(&v, p, 4);
  return v;
}

inline uint64_t hash_key(const uint8_t* p, int bits) {
  uint64_t a = load64(p) * 0x9E3779B97F4A7C15ull;
  uint64_t b = load64(p + 8) * 0xC2B2AE3D27D4EB4Full;
  uint64_t h = (a ^ ((b << 31) | (b >> 33))) * 0x165667B19E3779F9ull;
  return h >> (64 - bits);
}

inline uint32_t hash4(const uint8_t* p, int bits) { return (load32(p) * 2654435761u) >> (32 - bits); }

// length of the common prefix of a and b, at most limit (a precedes b)
inline uint64_t common(const uint8_t* a, const uint8_t* b, uint64_t limit) {
  uint64_t l = 0;
  while (l + 8 <= limit) {
    uint64_t x = load64(a + l) ^ load64(b + l);
    if (x) return l + (uint64_t)(__builtin_ctzll(x) >> 3);
    l += 8;
  }
  while (l < limit && a[l] == b[l]) l++;
  return l;
}

template <class F>
void parallel_for(uint64_t n, unsigned threads, F&& f) {
  if (threads <= 1 || n <= 1) {
    for (uint64_t i = 0; i < n; i++) f(i, 0u);
    return;
  }
  std::atomic<uint64_t> next{0};
  std::vector<std::thread> pool;
  unsigned t = (unsigned)std::min<uint64_t>(threads, n);
  for (unsigned k = 0; k < t; k++)
    pool.emplace_back([&, k] {
      for (uint64_t i; (i = next.fetch_add(1)) < n;) f(i, k);
    });
  for (auto& th : pool) th.join();
}

struct Token {
  uint32_t lit_run, match_len;
  uint64_t src;
};

// ------------------------------------------------------------- entropy layer

// f_s = max(1, floor(n_s 4096 / n)); shortfall to the most frequent symbol,
// excess taken one at a time from the largest frequency above 1.
void quantise(const uint8_t* sym, uint32_t n, uint32_t freq[256]) {
  uint64_t cnt[256] = {0};
  for (uint32_t i = 0; i < n; i++) cnt[sym[i]]++;
  int64_t sum = 0;
  int most = -1;
  for (int s = 0; s < 256; s++) {
    freq[s] = 0;
    if (!cnt[s]) continue;
    uint64_t f = std::max<uint64_t>(1, cnt[s] * ACE_SCALE / n);
    freq[s] = (uint32_t)f;
    sum += (int64_t)f;
    if (most < 0 || cnt[s] > cnt[most]) most = s;
  }
  if (sum < (int64_t)ACE_SCALE) freq[most] += (uint32_t)(ACE_SCALE - sum);
  while (sum > (int64_t)ACE_SCALE) {
    int big = -1;
    for (int s = 0; s < 256; s++)
      if (freq[s] > 1 && (big < 0 || freq[s] > freq[big])) big = s;
    freq[big]--;
    sum--;
  }
}

// Appends one 16-byte aligned stream payload for sym[0, n) to out.
void code_stream(const uint8_t* sym, uint32_t n, std::vector<uint8_t>& out) {
  if (n == 0) return;
  uint32_t freq[256], cum[256];
  quantise(sym, n, freq);
  uint32_t c = 0, present = 0;
  for (int s = 0; s < 256; s++) {
    cum[s] = c;
    c += freq[s];
    present += freq[s] != 0;
  }
  uint32_t x[ACE_NSTATES];
  for (auto& v : x) v = ACE_RANS_L;
  std::vector<uint8_t> rev;
  rev.reserve(n + 64);
  for (uint32_t i = n; i-- > 0;) {
    uint32_t s = sym[i], f = freq[s];
    uint32_t& xs = x[i & (ACE_NSTATES - 1)];
    uint64_t lim = (uint64_t)(ACE_RANS_L >> ACE_SCALE_BITS) << 8;
    lim *= f;
    while (xs >= lim) {
      rev.push_back((uint8_t)xs);
      xs >>= 8;
    }
    xs = ((xs / f) << ACE_SCALE_BITS) + (xs % f) + cum[s];
  }
  size_t base = out.size();
  size_t head = ACE_STREAM_HEAD + ((2 * (size_t)present + 15) & ~(size_t)15);
  out.resize(base + head + rev.size(), 0);
  uint8_t* p = out.data() + base;
  std::memcpy(p, x, sizeof x);
  uint32_t k = 0;
  for (int s = 0; s < 256; s++) {
    if (!freq[s]) continue;
    p[128 + s / 8] |= (uint8_t)(1u << (s % 8));
    p[ACE_STREAM_HEAD + 2 * k] = (uint8_t)freq[s];
    p[ACE_STREAM_HEAD + 2 * k + 1] = (uint8_t)(freq[s] >> 8);
    k++;
  }
  std::reverse_copy(rev.begin(), rev.end(), p + head);
}

// -------------------------------------------------------------- match layer

struct Global {
  std::vector<uint64_t> table;  // hash of a 16-byte key -> earliest position
  int bits = 0;
};

void build_global(const uint8_t* in, uint64_t n, unsigned threads, Global& g) {
  if (n < (uint64_t)kKey) return;
  uint64_t want = std::max<uint64_t>(1, n / kStride);
  int bits = 10;
  while (bits < 28 && (1ull << bits) < want) bits++;
  g.bits = bits;
  g.table.assign(1ull << bits, kEmpty);
  auto* tab = reinterpret_cast<std::atomic<uint64_t>*>(g.table.data());
  static_assert(sizeof(std::atomic<uint64_t>) == sizeof(uint64_t), "atomic layout");
  uint64_t last = n - kKey;  // last position whose key fits
  uint64_t nkeys = last / kStride + 1;
  uint64_t chunk = 1 << 16;
  uint64_t nchunks = (nkeys + chunk - 1) / chunk;
  parallel_for(nchunks, threads, [&](uint64_t c, unsigned) {
    uint64_t k1 = std::min(nkeys, (c + 1) * chunk);
    for (uint64_t k = c * chunk; k < k1; k++) {
      uint64_t q = k * kStride;
      std::atomic<uint64_t>& slot = tab[hash_key(in + q, bits)];
      uint64_t cur = slot.load(std::memory_order_relaxed);
      while (q < cur && !slot.compare_exchange_weak(cur, q, std::memory_order_relaxed)) {
      }
    }
  });
}

struct Parser {
  static constexpr int kHashBits = 15;
  std::vector<int32_t> head, prev;
  std::vector<uint8_t> wave;  // per block byte: the decoder's resolution wave (0: a literal)
  explicit Parser(uint32_t B) : head(1u << kHashBits), prev(B), wave(B) {}
};

// Where a block may take match sources from: its own earlier bytes, and
// earlier blocks outside its parse window whose dependency level is below the
// cap (so its own level stays at or below the cap).
struct Allowed {
  uint64_t window_start;        // first block of the current window
  const uint32_t* level;        // levels of the blocks before window_start
  uint32_t max_level;
  uint32_t log2B;
  // bytes from q that a match may read without entering a disallowed block
  uint64_t span(uint64_t q, uint64_t b, uint64_t want) const {
    uint64_t B = 1ull << log2B, k = q >> log2B, got = 0;
    while (got < want) {
      if (k != b && (k >= window_start || level[k] >= max_level)) break;
      uint64_t end = (k + 1) << log2B;
      got = std::min(want, end - q);
      k++;
      (void)B;
    }
    return got;
  }
};

void parse_block(const uint8_t* in, uint64_t n, uint64_t b, uint64_t bstart, uint64_t bend, uint32_t min_match,
                 uint32_t max_chain, const Global& g, const Allowed& al, Parser& ps, std::vector<Token>& toks) {
  std::fill(ps.head.begin(), ps.head.end(), -1);
  uint64_t gq[kStride];
  uint64_t gx[kStride];
  for (int j = 0; j < kStride; j++) gx[j] = kEmpty;
  auto global_at = [&](uint64_t x) -> uint64_t {  // earliest stride position sharing x's key
    int j = (int)(x % kStride);
    if (gx[j] != x) {
      gx[j] = x;
      gq[j] = (g.bits && x + kKey <= n) ? g.table[hash_key(in + x, g.bits)] : kEmpty;
    }
    return gq[j];
  };
  uint64_t inserted = bstart;
  auto insert_upto = [&](uint64_t p) {
    for (; inserted < p; inserted++) {
      if (inserted + 4 > bend) continue;
      uint32_t h = hash4(in + inserted, Parser::kHashBits);
      ps.prev[inserted - bstart] = ps.head[h];
      ps.head[h] = (int32_t)(inserted - bstart);
    }
  };
  // The decoder resolves a block's matches in waves: a match reading only
  // literals (or bytes of earlier blocks) resolves in wave 1, one reading
  // bytes written by wave-k matches in wave k + 1.  Candidates deeper than
  // kMaxWave are refused, and a shallower candidate within max(4, len/8)
  // bytes of the longest is preferred, so chains of match on match stay
  // short.  A source overlapping its own destination reads only [q, p).
  // Waves are 0..3, so the largest over a range is read from two bit tests
  // on the bytes, eight at a time: some byte 3 (both bits), else some byte
  // with bit 1 (a 2), else any non-zero byte (a 1).
  auto wave_of = [&](uint64_t q, uint64_t len, uint64_t p) -> uint32_t {
    static_assert(kMaxWave <= 3, "waves fit two bits");
    uint64_t lo = std::max(q, bstart), hi = std::min(q + len, p);
    const uint8_t* wv = ps.wave.data() - bstart;
    uint64_t any = 0, three = 0, k = lo;
    for (; k + 8 <= hi; k += 8) {
      const uint64_t x = load64(wv + k);
      any |= x;
      three |= x & (x >> 1);
    }
    for (; k < hi; k++) {
      const uint64_t x = wv[k];
      any |= x;
      three |= x & (x >> 1);
    }
    const uint32_t w = (three & 0x0101010101010101ull) ? 3u : (any & 0x0202020202020202ull) ? 2u : any ? 1u : 0u;
    return w + 1;
  };
  // the global table and the sources it names are random accesses: the
  // table slot of the key kAhead positions past the newest one looked up is
  // prefetched, and half as far ahead the slot is read and its source line
  // prefetched, so both are cached when the position is parsed
  constexpr uint64_t kAhead = 16;
  auto key_ok = [&](uint64_t x) { return g.bits && x + kKey <= n; };
  uint64_t p = bstart;
  uint32_t lit = 0;
  while (p < bend) {
    insert_upto(p);
    {
      const uint64_t xa = p + kStride - 1 + 2 * kAhead, xb = p + kStride - 1 + kAhead;
      if (key_ok(xa)) __builtin_prefetch(&g.table[hash_key(in + xa, g.bits)]);
      if (key_ok(xb)) {
        const uint64_t qq = g.table[hash_key(in + xb, g.bits)];
        if (qq != kEmpty && qq >= kStride) __builtin_prefetch(in + qq - kStride);
      }
    }
    uint64_t best_len = 0, best_q = 0;
    uint32_t best_w = 0;
    uint64_t room = bend - p;
    auto consider = [&](uint64_t q, uint64_t l) {
      if (l < min_match) return;
      uint64_t slack = std::max<uint64_t>(4, std::max(l, best_len) / 8);
      if (best_len && l + slack < best_len) return;  // too short to matter
      uint32_t w = wave_of(q, l, p);
      if (w > kMaxWave) return;
      bool take;
      if (!best_len) take = true;
      else if (w < best_w) take = l + slack >= best_len;                // shallower, nearly as long
      else if (w > best_w) take = l > best_len + std::max<uint64_t>(4, l / 8);  // deeper: only if clearly longer
      else take = l > best_len || (l == best_len && q < best_q);
      if (take) {
        best_len = l;
        best_q = q;
        best_w = w;
      }
    };
    if (room >= min_match) {
      if (p + 4 <= bend) {  // repeats inside the block, most recent first
        uint32_t depth = 0;
        int32_t r = ps.head[hash4(in + p, Parser::kHashBits)];
        for (; r >= 0 && depth < max_chain; r = ps.prev[r], depth++) {
          uint64_t q = bstart + (uint64_t)r;
          consider(q, common(in + q, in + p, room));
        }
        // past the usual depth, look further back for a shallower source
        for (uint32_t extra = 0; r >= 0 && extra < 16 * max_chain && best_w > 1; r = ps.prev[r], extra++) {
          uint64_t q = bstart + (uint64_t)r;
          consider(q, common(in + q, in + p, room));
        }
      }
      uint64_t tried[kStride];
      int nt = 0;
      for (int j = 0; j < kStride; j++) {  // earliest occurrence anywhere before p
        uint64_t qq = global_at(p + (uint64_t)j);
        if (qq == kEmpty || qq < (uint64_t)j) continue;
        uint64_t q = qq - (uint64_t)j;
        if (q >= p) continue;
        bool seen = false;  // keys of one earlier occurrence name the same source
        for (int t = 0; t < nt; t++) seen |= tried[t] == q;
        if (seen) continue;
        tried[nt++] = q;
        uint64_t l = common(in + q, in + p, room);
        if (q < bstart) l = al.span(q, b, l);
        consider(q, l);
      }
    }
    if (best_len >= min_match) {
      toks.push_back({lit, (uint32_t)best_len, best_q});
      lit = 0;
      for (uint64_t k = p; k < p + best_len; k++) ps.wave[k - bstart] = (uint8_t)best_w;
      p += best_len;
    } else {
      ps.wave[p - bstart] = 0;
      lit++;
      p++;
    }
  }
  toks.push_back({lit, 0, 0});
}

// ------------------------------------------------------------ block coding

struct BlockOut {
  std::vector<uint8_t> payload;   // three streams, each padded to 16 bytes
  uint32_t stream_bytes[3] = {0, 0, 0};
  uint32_t nsym[3] = {0, 0, 0};
  uint8_t mode[3] = {0, 0, 0};    // 0: rANS, 1: stored verbatim
  uint32_t ntok = 0, nesc = 0;
  std::vector<uint32_t> deps;     // (first, last) pairs
  uint64_t n_matches = 0, match_bytes = 0, match_src_bytes = 0;
};

void code_block(const uint8_t* in, uint64_t b, uint64_t B, uint64_t n, int w, const std::vector<Token>& toks,
                bool adaptive, BlockOut& bo) {
  std::vector<uint8_t> lit, esc, codes, off;
  uint64_t bstart = b * B, dst = bstart;
  std::vector<std::pair<uint64_t, uint64_t>> rg;
  for (size_t t = 0; t < toks.size(); t++) {
    const Token& tk = toks[t];
    lit.insert(lit.end(), in + dst, in + dst + tk.lit_run);
    dst += tk.lit_run;
    for (uint32_t v : {tk.lit_run, tk.match_len}) {
      if (v < 255) {
        codes.push_back((uint8_t)v);
      } else {
        codes.push_back(255);
        esc.push_back((uint8_t)(v - 255));
        esc.push_back((uint8_t)((v - 255) >> 8));
      }
    }
    if (t + 1 < toks.size()) {
      for (int k = 0; k < w; k++) off.push_back((uint8_t)(tk.src >> (8 * k)));
      uint64_t rl = std::min<uint64_t>(tk.match_len, dst - tk.src);
      bo.n_matches += tk.match_len != 0;
      bo.match_bytes += tk.match_len;
      bo.match_src_bytes += rl;
      uint64_t f = tk.src / B, l = (tk.src + rl - 1) / B;
      if (l >= b) l = b - 1;
      if (f < b && f <= l) rg.push_back({f, l});
    }
    dst += tk.match_len;
  }
  (void)n;
  std::sort(rg.begin(), rg.end());
  for (size_t i = 0; i < rg.size();) {
    uint64_t f = rg[i].first, l = rg[i].second;
    size_t j = i + 1;
    while (j < rg.size() && rg[j].first <= l + 1) l = std::max(l, rg[j++].second);
    bo.deps.push_back((uint32_t)f);
    bo.deps.push_back((uint32_t)l);
    i = j;
  }
  std::vector<uint8_t> lens(esc);
  lens.insert(lens.end(), codes.begin(), codes.end());
  const std::vector<uint8_t>* st[3] = {&lit, &lens, &off};
  for (int k = 0; k < 3; k++) {
    size_t before = bo.payload.size();
    code_stream(st[k]->data(), (uint32_t)st[k]->size(), bo.payload);
    bo.stream_bytes[k] = (uint32_t)(bo.payload.size() - before);
    if (adaptive && !st[k]->empty() && bo.stream_bytes[k] >= st[k]->size()) {
      // rANS did not shrink the stream (its fixed head outweighs the gain on
      // short or near-uniform streams): store the symbols verbatim
      bo.payload.resize(before);
      bo.payload.insert(bo.payload.end(), st[k]->begin(), st[k]->end());
      bo.stream_bytes[k] = (uint32_t)st[k]->size();
      bo.mode[k] = 1;
    }
    bo.payload.resize((bo.payload.size() + 15) & ~(size_t)15, 0);
    bo.nsym[k] = (uint32_t)st[k]->size();
  }
  bo.ntok = (uint32_t)toks.size();
  bo.nesc = (uint32_t)(esc.size() / 2);
}

}  // namespace

struct ace_encoder {
  ace_file_header hdr{};
  std::vector<ace_block_dir> dir;
  std::vector<uint32_t> dep_ptr, dep_iv;
  std::vector<BlockOut> blocks;
  std::vector<uint64_t> block_pos;  // payload offset of each block, relative to payload_off
  ace_encode_stats stats{};
};

extern "C" {

ace_status ace_encode_bound(uint64_t n, uint32_t log2_block, uint64_t* bound) {
  if (!bound || log2_block < ACE_MIN_LOG2_BLOCK || log2_block > ACE_MAX_LOG2_BLOCK) return ACE_E_INVAL;
  uint64_t B = 1ull << log2_block, nb = (n + B - 1) / B;
  // per block: streams <= 2 bytes per symbol plus heads, symbols <= 2.8 B;
  // dependency pairs <= B/4 + 1; directory 64 bytes
  *bound = 1024 + 4 * (nb + 1) + nb * (9 * B + 4096);
  return ACE_OK;
}

ace_status ace_encode_run(const void* h_in, uint64_t n, const ace_encode_params* prm, ace_encoder** out,
                          uint64_t* arc_len) {
  if (!prm || !out || !arc_len || (n && !h_in)) return ACE_E_INVAL;
  if (prm->log2_block < ACE_MIN_LOG2_BLOCK || prm->log2_block > ACE_MAX_LOG2_BLOCK || prm->min_match < 4)
    return ACE_E_INVAL;
  const uint8_t* in = static_cast<const uint8_t*>(h_in);
  unsigned threads = prm->threads ? prm->threads : std::max(1u, std::thread::hardware_concurrency());
  uint32_t max_chain = prm->max_chain ? prm->max_chain : 16;
  uint32_t max_level = kMaxLevel;
  uint64_t B = 1ull << prm->log2_block, nb = (n + B - 1) / B;
  if (nb > 0xFFFFFFFFull) return ACE_E_INVAL;
  if (prm->off_width != 0 && prm->off_width != 4 && prm->off_width != 5) return ACE_E_INVAL;
  if (prm->adaptive > 1) return ACE_E_INVAL;
  if (prm->off_width == 4 && n > (1ull << 32)) return ACE_E_INVAL;
  int w = (n > (1ull << 32) || prm->off_width == 5) ? 5 : 4;
  ace_encoder* e = new (std::nothrow) ace_encoder();
  if (!e) return ACE_E_NOMEM;
  try {
    Global g;
    build_global(in, n, threads, g);
    e->blocks.resize(nb);
    std::vector<uint32_t> level(nb, 0);
    std::vector<Parser*> parsers(threads, nullptr);
    for (uint64_t w0 = 0; w0 < nb; w0 += kWindow) {
      uint64_t w1 = std::min(nb, w0 + kWindow);
      Allowed al{w0, level.data(), max_level, prm->log2_block};
      parallel_for(w1 - w0, threads, [&](uint64_t i, unsigned k) {
        uint64_t b = w0 + i;
        if (!parsers[k]) parsers[k] = new Parser((uint32_t)B);
        std::vector<Token> toks;
        uint64_t bstart = b * B, bend = std::min(n, bstart + B);
        parse_block(in, n, b, bstart, bend, prm->min_match, max_chain, g, al, *parsers[k], toks);
        code_block(in, b, B, n, w, toks, prm->adaptive != 0, e->blocks[b]);
      });
      for (uint64_t b = w0; b < w1; b++) {  // level: 1 + the deepest block read
        const std::vector<uint32_t>& dv = e->blocks[b].deps;
        uint32_t lv = 0;
        for (size_t i = 0; i < dv.size(); i += 2)
          for (uint32_t k = dv[i]; k <= dv[i + 1]; k++) lv = std::max(lv, level[k] + 1);
        level[b] = lv;
      }
    }
    for (auto* p : parsers) delete p;
    uint32_t maxlv = 0;
    for (uint64_t b = 0; b < nb; b++) maxlv = std::max(maxlv, level[b]);
    e->stats.n_levels = nb ? maxlv + 1 : 0;
  } catch (const std::bad_alloc&) {
    delete e;
    return ACE_E_NOMEM;
  }
  // layout: header | directory | dependency table | payload
  e->dir.assign(nb, ace_block_dir{});
  e->dep_ptr.resize(nb + 1);
  e->block_pos.resize(nb);
  uint64_t niv = 0, pos = 0;
  for (uint64_t b = 0; b < nb; b++) {
    BlockOut& bo = e->blocks[b];
    e->dep_ptr[b] = (uint32_t)niv;
    niv += bo.deps.size() / 2;
    e->block_pos[b] = pos;
    ace_block_dir& d = e->dir[b];
    uint64_t s = pos;
    for (int k = 0; k < 3; k++) {
      d.stream_off[k] = s;
      d.stream_bytes[k] = bo.stream_bytes[k];
      d.nsym[k] = bo.nsym[k];
      d.mode[k] = bo.mode[k];
      s += (bo.stream_bytes[k] + 15) & ~15ull;
    }
    d.ntok = bo.ntok;
    d.nesc = bo.nesc;
    e->stats.n_tokens += bo.ntok;
    e->stats.n_matches += bo.n_matches;
    e->stats.literal_bytes += bo.nsym[ACE_S_LIT];
    e->stats.match_bytes += bo.match_bytes;
    e->stats.match_src_bytes += bo.match_src_bytes;
    pos += bo.payload.size();
  }
  e->dep_ptr[nb] = (uint32_t)niv;
  e->stats.n_dep_intervals = niv;
  e->dep_iv.reserve(2 * niv);
  for (uint64_t b = 0; b < nb; b++) e->dep_iv.insert(e->dep_iv.end(), e->blocks[b].deps.begin(), e->blocks[b].deps.end());
  ace_file_header& h = e->hdr;
  h.magic = ACE_MAGIC;
  h.version = ACE_VERSION;
  h.n_streams = ACE_NSTREAMS;
  h.n_states = ACE_NSTATES;
  h.scale_bits = ACE_SCALE_BITS;
  h.off_width = (uint8_t)w;
  h.log2_block = (uint8_t)prm->log2_block;
  h.total_size = n;
  h.n_blocks = nb;
  h.dir_off = sizeof(ace_file_header);
  h.deps_off = h.dir_off + nb * sizeof(ace_block_dir);
  h.payload_off = (h.deps_off + 4 * (nb + 1) + 8 * niv + 15) & ~15ull;
  h.archive_bytes = (h.payload_off + pos + 15) & ~15ull;
  *out = e;
  *arc_len = h.archive_bytes;
  return ACE_OK;
}

ace_status ace_encode_write(const ace_encoder* e, void* h_arc, uint64_t cap) {
  if (!e || !h_arc) return ACE_E_INVAL;
  const ace_file_header& h = e->hdr;
  if (cap < h.archive_bytes) return ACE_E_NOMEM;
  uint8_t* a = static_cast<uint8_t*>(h_arc);
  std::memset(a, 0, h.payload_off);
  std::memcpy(a, &h, sizeof h);
  std::memcpy(a + h.dir_off, e->dir.data(), e->dir.size() * sizeof(ace_block_dir));
  std::memcpy(a + h.deps_off, e->dep_ptr.data(), e->dep_ptr.size() * 4);
  std::memcpy(a + h.deps_off + 4 * e->dep_ptr.size(), e->dep_iv.data(), e->dep_iv.size() * 4);
  unsigned threads = std::max(1u, std::thread::hardware_concurrency());
  parallel_for(e->blocks.size(), threads, [&](uint64_t b, unsigned) {
    const BlockOut& bo = e->blocks[b];
    std::memcpy(a + h.payload_off + e->block_pos[b], bo.payload.data(), bo.payload.size());
  });
  uint64_t end = h.payload_off + (e->blocks.empty() ? 0 : e->block_pos.back() + e->blocks.back().payload.size());
  std::memset(a + end, 0, h.archive_bytes - end);
  return ACE_OK;
}

ace_status ace_encode_get_stats(const ace_encoder* e, ace_encode_stats* st) {
  if (!e || !st) return ACE_E_INVAL;
  *st = e->stats;
  return ACE_OK;
}

ace_status ace_encode_free(ace_encoder* e) {
  delete e;
  return ACE_OK;
}

ace_status ace_encode(const void* h_in, uint64_t n, const ace_encode_params* prm, void* h_arc, uint64_t cap,
                      uint64_t* arc_len) {
  ace_encoder* e = nullptr;
  ace_status rc = ace_encode_run(h_in, n, prm, &e, arc_len);
  if (rc != ACE_OK) return rc;
  rc = ace_encode_write(e, h_arc, cap);
  ace_encode_free(e);
  return rc;
}

}  // extern "C"
