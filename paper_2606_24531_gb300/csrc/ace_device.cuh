// Device-side building blocks of the decoder: status reporting, bounded
// waits, per-stream rANS state and lookup tables, warp scans.
#pragma once
#include <cstdint>

#include "ace.h"
#include "ace_format.h"

namespace ace {

constexpr uint32_t kFull = 0xffffffffu;
constexpr uint32_t kLanes = 32;

// First 256 bytes of every scratch buffer.
struct ScratchHdr {
  uint32_t status;     // first device-side error (ace_status), 0 when none
  uint32_t err_block;  // block that recorded it
  uint32_t err_where;  // which check fired (diagnostics)
  uint32_t epoch;      // value a block's ready flag takes when it is published
  uint32_t ticket;     // next work item handed to a persistent warp
  uint32_t n_work;     // seek: blocks in the work list
  uint32_t n_front;    // seek: frontier size during the closure search
  uint32_t min_block;  // seek: smallest block reached by the closure
  uint64_t fnv;        // verify: last FNV-1a 64 computed
  uint64_t guard_bad;  // verify: guard bytes that differ from the canary
  uint32_t ticket2;    // next work item of the literal pass
  uint32_t ticket3;    // next work item of the match pass
  uint32_t lv_start[33];  // seek by levels: the work list's level l is [lv_start[l], lv_start[l + 1])
  uint32_t pad[17];
};
static_assert(sizeof(ScratchHdr) == 256, "scratch header");

// First 256 bytes of the index memory.
struct IndexHdr {
  uint32_t status;
  uint32_t err_block;
  uint32_t err_where;
  uint32_t n_levels;
  uint32_t max_ntok;   // most tokens in any block: sizes a seek slot's match records
  uint32_t pad0;
  uint64_t n_matches;  // matches in the archive: sizes a whole decode's match records
  uint32_t relax[8];   // level sweep k changed a level
  uint32_t n_iv;       // dependency intervals in the archive
  uint32_t lvc[33];    // blocks per level, for the first 33 levels
  uint32_t pad[14];
};
static_assert(sizeof(IndexHdr) == 256, "index header");

// One match of a block, between the token pass that finds it and the match
// pass that resolves it: absolute source, destination within the block,
// length.
struct MatchRec {
  uint64_t S;
  uint32_t D;
  uint32_t L;
};
static_assert(sizeof(MatchRec) == 16, "match record");

// One stream's decode tables: slot -> symbol, and symbol -> (freq << 16 | cum).
struct Lut {
  uint8_t sym[ACE_SCALE];
  uint32_t fc[256];
};

__device__ __forceinline__ void record_error(uint32_t* status, uint32_t* err_block, uint32_t* err_where,
                                             ace_status code, uint32_t block, uint32_t where) {
  if (atomicCAS(status, 0u, (uint32_t)code) == 0u) {
    *err_block = block;
    *err_where = where;
  }
}

__device__ __forceinline__ uint64_t globaltimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

// A relaxed load: independent ones overlap in flight.  Followed by
// fence_acquire() once it has observed a released value, it acquires.
__device__ __forceinline__ uint32_t ld_relaxed(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void fence_acquire() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }

__device__ __forceinline__ uint32_t ld_acquire(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_release(uint32_t* p, uint32_t v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Spins until *flag == want or timeout_ns passes; false on timeout.
// Gives up after timeout_ns, or as soon as *abort (a call's status word)
// records an error: the block waited for may then never be published.
__device__ __forceinline__ bool wait_flag(const uint32_t* flag, uint32_t want, uint64_t timeout_ns,
                                          const uint32_t* abort = nullptr) {
  if (ld_acquire(flag) == want) return true;
  uint64_t t0 = globaltimer();
  uint32_t ns = 32;
  while (true) {
    __nanosleep(ns);
    if (ld_acquire(flag) == want) return true;
    if (globaltimer() - t0 > timeout_ns) return false;
    if (abort && *(volatile const uint32_t*)abort) return false;
    if (ns < 1024) ns <<= 1;
  }
}

__device__ __forceinline__ uint32_t lanemask_lt() {
  uint32_t m;
  asm("mov.u32 %0, %lanemask_lt;" : "=r"(m));
  return m;
}

__device__ __forceinline__ uint32_t warp_incl_sum(uint32_t v, uint32_t lane) {
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    uint32_t u = __shfl_up_sync(kFull, v, d);
    if (lane >= (uint32_t)d) v += u;
  }
  return v;
}

__device__ __forceinline__ uint32_t warp_excl_max(uint32_t v, uint32_t lane) {
  uint32_t incl = v;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    uint32_t u = __shfl_up_sync(kFull, incl, d);
    if (lane >= (uint32_t)d) incl = max(incl, u);
  }
  uint32_t ex = __shfl_up_sync(kFull, incl, 1);
  return lane ? ex : 0u;
}

__device__ __forceinline__ uint32_t warp_min(uint32_t v) {
#pragma unroll
  for (int d = 16; d; d >>= 1) v = min(v, __shfl_xor_sync(kFull, v, d));
  return v;
}

__device__ __forceinline__ uint64_t warp_min64(uint64_t v) {
#pragma unroll
  for (int d = 16; d; d >>= 1) {
    uint64_t u = __shfl_xor_sync(kFull, v, d);
    v = u < v ? u : v;
  }
  return v;
}

// ----------------------------------------------------------- async copies

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  uint32_t d = (uint32_t)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// ------------------------------------------------------- one rANS stream

// Renormalisation bytes reach the decoder through a 512-byte ring in shared
// memory: four 128-byte segments, each refilled with cp.async as soon as it
// has been consumed, so the byte loads on the decode chain hit shared memory.
constexpr uint32_t kRing = 512;
constexpr uint32_t kSeg = 128;

// State of one interleaved-rANS stream decoded by one warp: lane j holds the
// state of interleaved lane j; every other field is warp-uniform.
struct Stream {
  const uint8_t* g;    // renormalisation bytes (16-byte aligned); the payload starts head bytes before
  uint32_t head;       // bytes of states, present bitmap and frequencies
  uint32_t k;          // search mode: present symbols (0: slot table mode)
  uint32_t nsym;       // symbols in the stream
  uint32_t nbytes;     // renormalisation bytes
  uint32_t next;       // next symbol index to decode
  uint32_t pos;        // renormalisation bytes consumed
  uint32_t base;       // renormalisation offset held by the ring's oldest segment
  uint32_t x;          // this lane's state
  uint32_t stored;     // mode 1: the stream holds its symbols verbatim at g (no states, no table)
};

// Copies renormalisation bytes [off, off + 128) into their segment of a
// RING-byte ring; the copyable extent is nbytes rounded up to 16, which stays
// inside the archive.  A ring of RING / 128 segments keeps all but the two
// newest landed (the refill waits for the rest).
template <uint32_t RING = kRing>
__device__ __forceinline__ void ring_issue(const Stream& st, uint8_t* ring, uint32_t off, uint32_t lane) {
  static_assert(RING % kSeg == 0 && (RING & (RING - 1)) == 0 && RING / kSeg >= 4, "ring of segments");
  uint32_t o = off + 16 * lane;
  if (lane < kSeg / 16 && o < ((st.nbytes + 15) & ~15u)) cp_async16(ring + (o & (RING - 1)), st.g + o);
  cp_async_commit();
}

// Reads the entry states (Section 3: the block boundary is the entropy entry
// point) and locates the renormalisation bytes; issues the first ring fill.
// The stream bounds were validated when the index was built.  Returns false
// (all lanes) for a state outside [L, 2^31) or a table overrunning the stream.
//
// A stored stream (mode 1; entropy coding chosen per stream at encode time)
// has no states or table: its bytes are its symbols, read straight from the
// archive, so it opens with nothing to check but its length.
template <uint32_t RING = kRing>
__device__ __forceinline__ bool stream_open(const uint8_t* pay, uint32_t sbytes, uint32_t nsym, uint8_t* ring,
                                            Stream& st, uint32_t lane, uint32_t mode = 0) {
  st.nsym = nsym;
  st.next = st.pos = st.base = 0;
  st.x = ACE_RANS_L;
  st.g = pay;
  st.head = 0;
  st.k = 0;
  st.nbytes = 0;
  st.stored = mode == 1;
  if (nsym == 0) return sbytes == 0;
  if (st.stored) {
    st.nbytes = sbytes;
    return sbytes == nsym;
  }
  uint32_t x = reinterpret_cast<const uint32_t*>(pay)[lane];
  uint32_t present = __popc(pay[128 + lane]);
  present = warp_incl_sum(present, lane);
  present = __shfl_sync(kFull, present, 31);
  uint32_t head = ACE_STREAM_HEAD + ((2 * present + 15) & ~15u);
  bool bad = x < ACE_RANS_L || x >= (1u << 31) || head > sbytes;
  if (__any_sync(kFull, bad)) return false;
  st.x = x;
  st.g = pay + head;
  st.head = head;
  st.nbytes = sbytes - head;
  for (uint32_t s = 0; s < RING / kSeg; s++) ring_issue<RING>(st, ring, s * kSeg, lane);
  // the frequency table (bytes 160 .. head) is read when the stream's tables
  // are built: bring its lines into L1 now
  if (lane < 5 && 128 + 128 * lane < head) {
    const uint8_t* line = pay + 128 + 128 * lane;
    asm volatile("prefetch.global.L1 [%0];" ::"l"(line));
  }
  return true;
}

// Streams of at most kSearchMaxSymbols symbols are decoded by looking their
// symbols up among the present ones (a coarse table of bucket owners, then a
// short forward step) instead of building the 4096-entry slot table, whose
// build costs more than such a stream's rounds save (measured on the FASTQ,
// genome and text token streams and on batches of 4-64 KiB blocks).
constexpr uint32_t kSearchMaxSymbols = 2048;
constexpr uint32_t kCoarseOff = 1024;  // search mode: the coarse table after the (at most 256) packed words

// Builds the stream's decode tables.  Slot table mode: fc[s] = f_s << 16 |
// c_s, and the slot -> symbol table by marking each symbol's first slot and
// taking a prefix maximum (symbols increase with their slots).  Search mode
// (short streams): one sorted word per present symbol, c << 20 | (f - 1) << 8
// | s, searched per symbol.  Returns false (all lanes) if the frequencies do
// not sum to 4096.
__device__ __forceinline__ bool lut_build(Stream& st, Lut& lut, uint32_t lane) {
  if (st.nsym == 0 || st.stored) return true;
  const uint8_t* sp = st.g - st.head;
  uint32_t bm = sp[128 + lane];
  uint32_t cnt = __popc(bm);
  uint32_t first = warp_incl_sum(cnt, lane) - cnt;
  uint32_t f[8], fsum = 0;
  const uint8_t* fp = sp + ACE_STREAM_HEAD;
  uint32_t k = first;
  bool bad = false;
#pragma unroll
  for (int j = 0; j < 8; j++) {
    f[j] = 0;
    if ((bm >> j) & 1) {
      f[j] = (uint32_t)fp[2 * k] | ((uint32_t)fp[2 * k + 1] << 8);
      k++;
      bad |= f[j] == 0 || f[j] > ACE_SCALE;
    }
    fsum += f[j];
  }
  uint32_t cincl = warp_incl_sum(fsum, lane);
  bad |= __shfl_sync(kFull, cincl, 31) != ACE_SCALE;
  if (__any_sync(kFull, bad)) return false;
  const uint32_t present = __shfl_sync(kFull, first + cnt, 31);  // present symbols
  if (st.nsym <= kSearchMaxSymbols) {
    // the packed words, and beside them the coarse table: entry b is the
    // index of the symbol owning slot 16 b.  Each symbol marks the first
    // bucket start in its range; a prefix maximum carries the mark over the
    // rest of the range (indices grow with slots, and slot 0 is marked).
    uint32_t* pk = reinterpret_cast<uint32_t*>(lut.sym);
    uint8_t* cz = lut.sym + kCoarseOff;
    reinterpret_cast<uint2*>(cz)[lane] = make_uint2(0u, 0u);
    __syncwarp();
    uint32_t c = cincl - fsum, j = first;
#pragma unroll
    for (int q = 0; q < 8; q++)
      if (f[q]) {
        pk[j] = (c << 20) | ((f[q] - 1) << 8) | (lane * 8 + q);
        const uint32_t bb = (c + 15) >> 4;  // the first bucket starting in [c, c + f)
        if (16 * bb < c + f[q]) cz[bb] = (uint8_t)j;
        j++;
        c += f[q];
      }
    __syncwarp();
    uint2 w = reinterpret_cast<uint2*>(cz)[lane];  // entries 8 lane .. 8 lane + 7
    w.x = __vmaxu4(w.x, w.x << 8);
    w.x = __vmaxu4(w.x, w.x << 16);
    w.y = __vmaxu4(w.y, w.y << 8);
    w.y = __vmaxu4(__vmaxu4(w.y, w.y << 16), (w.x >> 24) * 0x01010101u);
    const uint32_t carry = warp_excl_max(w.y >> 24, lane);
    w.x = __vmaxu4(w.x, carry * 0x01010101u);
    w.y = __vmaxu4(w.y, carry * 0x01010101u);
    reinterpret_cast<uint2*>(cz)[lane] = w;
    st.k = present;
    __syncwarp();
    return true;
  }
  st.k = 0;
  uint4* sym4 = reinterpret_cast<uint4*>(lut.sym);
#pragma unroll
  for (int j = 0; j < 8; j++) sym4[lane * 8 + j] = make_uint4(0, 0, 0, 0);
  __syncwarp();
  uint32_t c = cincl - fsum;
#pragma unroll
  for (int j = 0; j < 8; j++) {
    uint32_t s = lane * 8 + j;
    lut.fc[s] = f[j] ? ((f[j] << 16) | c) : 0u;
    if (f[j]) lut.sym[c] = (uint8_t)s;
    c += f[j];
  }
  __syncwarp();
  uint4 w[8];
  uint32_t lmax = 0;
#pragma unroll
  for (int j = 0; j < 8; j++) {
    w[j] = sym4[lane * 8 + j];
    lmax = __vmaxu4(lmax, __vmaxu4(__vmaxu4(w[j].x, w[j].y), __vmaxu4(w[j].z, w[j].w)));
  }
  lmax = max(max(lmax & 0xff, (lmax >> 8) & 0xff), max((lmax >> 16) & 0xff, lmax >> 24));
  uint32_t carry = warp_excl_max(lmax, lane);
#pragma unroll
  for (int j = 0; j < 8; j++) {
    uint32_t* ww = reinterpret_cast<uint32_t*>(&w[j]);
#pragma unroll
    for (int q = 0; q < 4; q++) {
      uint32_t m = __vmaxu4(ww[q], ww[q] << 8);
      m = __vmaxu4(m, m << 16);
      m = __vmaxu4(m, carry * 0x01010101u);
      carry = m >> 24;
      ww[q] = m;
    }
    sym4[lane * 8 + j] = w[j];
  }
  __syncwarp();
  return true;
}

// The symbol owning a slot, with its frequency and cumulative frequency.
__device__ __forceinline__ void lookup(const Stream& st, const Lut& lut, uint32_t slot, uint32_t& s, uint32_t& f,
                                       uint32_t& c) {
  if (st.k) {
    const uint32_t* pk = reinterpret_cast<const uint32_t*>(lut.sym);
    uint32_t lo = lut.sym[kCoarseOff + (slot >> 4)];  // owner of the bucket's first slot
    while (lo + 1 < st.k && (pk[lo + 1] >> 20) <= slot) lo++;  // at most 15 starts inside a bucket
    uint32_t e = pk[lo];
    s = e & 0xffu;
    f = ((e >> 8) & 0xfffu) + 1;
    c = e >> 20;
  } else {
    s = lut.sym[slot];
    uint32_t fc = lut.fc[s];
    f = fc >> 16;
    c = fc & 0xffffu;
  }
}

// Decodes one round of up to 32 symbols of [st.next, end): symbol i is on
// lane i mod 32 (interleaved rANS).  slot = x mod 4096, s = sym[slot],
// x <- f_s floor(x / 4096) + slot - c_s; then x takes k in {0,1,2} bytes,
// k = [x < 2^23] + [x < 2^15].  Bytes are consumed in symbol order, so lane j
// reads at the running position plus the bytes of lower lanes, high byte
// first.  Branch-free: every lane fetches the two candidate bytes and
// selects.  Bytes read past the end of the stream come from the ring and are
// harmless; the end-of-stream check (all bytes consumed, every state at L)
// rejects a stream that needed them.  Sets act and i for this lane and
// returns the symbol.
template <uint32_t RING = kRing>
__device__ __forceinline__ uint32_t rans_round(Stream& st, uint8_t* ring, const Lut& lut, uint32_t end,
                                               uint32_t lane, uint32_t lt, bool& act, uint32_t& i) {
  if (st.pos >= st.base + kSeg) {  // oldest segment consumed: refill it further on
    ring_issue<RING>(st, ring, st.base + RING, lane);
    st.base += kSeg;
    cp_async_wait<RING / kSeg - 2>();
    __syncwarp();
  }
  uint32_t base = st.next & ~31u;
  i = base + lane;
  act = i >= st.next && i < end;
  uint32_t x = st.x;
  uint32_t slot = x & (ACE_SCALE - 1);
  uint32_t s, f, c;
  lookup(st, lut, slot, s, f, c);
  uint32_t xn = f * (x >> ACE_SCALE_BITS) + slot - c;
  bool p1 = act && xn < ACE_RANS_L, p2 = act && xn < (1u << 15);
  uint32_t b1 = __ballot_sync(kFull, p1), b2 = __ballot_sync(kFull, p2);
  uint32_t p = st.pos + __popc(b1 & lt) + __popc(b2 & lt);
  uint32_t c0 = ring[p & (RING - 1)], c1 = ring[(p + 1) & (RING - 1)];
  uint32_t x1 = (xn << 8) | c0, x2 = (x1 << 8) | c1;
  xn = p2 ? x2 : (p1 ? x1 : xn);
  st.x = act ? xn : x;
  st.pos += __popc(b1) + __popc(b2);
  st.next = min(base + 32, end);
  return s;
}

// A full round: st.next is a multiple of 32 and at least 32 symbols remain,
// so every lane is active.
template <uint32_t RING = kRing>
__device__ __forceinline__ uint32_t rans_round_full(Stream& st, uint8_t* ring, const Lut& lut, uint32_t lt) {
  if (st.pos >= st.base + kSeg) {
    ring_issue<RING>(st, ring, st.base + RING, threadIdx.x & 31);
    st.base += kSeg;
    cp_async_wait<RING / kSeg - 2>();
    __syncwarp();
  }
  uint32_t x = st.x;
  uint32_t slot = x & (ACE_SCALE - 1);
  uint32_t s, f, c;
  lookup(st, lut, slot, s, f, c);
  uint32_t xn = f * (x >> ACE_SCALE_BITS) + slot - c;
  bool p1 = xn < ACE_RANS_L, p2 = xn < (1u << 15);
  uint32_t b1 = __ballot_sync(kFull, p1);
  if (!__any_sync(kFull, p2)) {
    uint32_t c0 = ring[(st.pos + __popc(b1 & lt)) & (RING - 1)];
    st.x = p1 ? ((xn << 8) | c0) : xn;
    st.pos += __popc(b1);
  } else {
    uint32_t b2 = __ballot_sync(kFull, p2);
    uint32_t p = st.pos + __popc(b1 & lt) + __popc(b2 & lt);
    uint32_t c0 = ring[p & (RING - 1)], c1 = ring[(p + 1) & (RING - 1)];
    uint32_t x1 = (xn << 8) | c0, x2 = (x1 << 8) | c1;
    st.x = p2 ? x2 : (p1 ? x1 : xn);
    st.pos += __popc(b1) + __popc(b2);
  }
  st.next += 32;
  return s;
}

// Decodes symbols [st.next, end), handing each to sink(act, i, s) per
// round (act false on lanes without a symbol this round): a partial first
// round up to the next multiple of 32, full rounds, then a partial last one.
template <uint32_t RING = kRing, class Sink>
__device__ __forceinline__ void rans_run(Stream& st, uint8_t* ring, const Lut& lut, uint32_t end, uint32_t lane,
                                         uint32_t lt, Sink&& sink) {
  if (st.stored) {  // symbol i is byte i, in rounds of 32 like the coded streams
    while (st.next < end) {
      const uint32_t base = st.next & ~31u, i = base + lane;
      const bool act = i >= st.next && i < end;
      const uint32_t s = act ? (uint32_t)__ldg(st.g + i) : 0u;
      sink(act, i, s);
      st.next = min(base + 32, end);
    }
    st.pos = st.next;  // a stored stream's bytes are consumed one per symbol
    return;
  }
  if (st.next < end && ((st.next & 31) || end - st.next < 32)) {
    bool act;
    uint32_t i;
    uint32_t s = rans_round<RING>(st, ring, lut, end, lane, lt, act, i);
    sink(act, i, s);
  }
  while (end - st.next >= 32 && st.next < end) {
    uint32_t i = st.next + lane;
    uint32_t s = rans_round_full<RING>(st, ring, lut, lt);
    sink(true, i, s);
  }
  if (st.next < end) {
    bool act;
    uint32_t i;
    uint32_t s = rans_round<RING>(st, ring, lut, end, lane, lt, act, i);
    sink(act, i, s);
  }
}

// One full round in slot-table mode (st.k == 0): every lane decodes one
// symbol of state x, with renormalisation bytes read from the ring at the
// running position pos as in rans_round.  The caller checks the ring.
template <uint32_t RING = kRing>
__device__ __forceinline__ uint32_t table_round(uint32_t& x, uint32_t& pos, const uint8_t* ring, const Lut& lut,
                                                uint32_t lt) {
  const uint32_t slot = x & (ACE_SCALE - 1);
  const uint32_t s = lut.sym[slot];
  const uint32_t fc = lut.fc[s];
  const uint32_t xn = (fc >> 16) * (x >> ACE_SCALE_BITS) + slot - (fc & 0xffffu);
  const bool p1 = xn < ACE_RANS_L, p2 = xn < (1u << 15);
  const uint32_t b1 = __ballot_sync(kFull, p1);
  if (!__any_sync(kFull, p2)) {  // no state takes two bytes (most rounds): one read per lane
    const uint32_t p = pos + __popc(b1 & lt);
    const uint32_t c0 = ring[p & (RING - 1)];
    x = p1 ? ((xn << 8) | c0) : xn;
    pos += __popc(b1);
  } else {
    const uint32_t b2 = __ballot_sync(kFull, p2);
    const uint32_t p = pos + __popc(b1 & lt) + __popc(b2 & lt);
    const uint32_t c0 = ring[p & (RING - 1)], c1 = ring[(p + 1) & (RING - 1)];
    const uint32_t x1 = (xn << 8) | c0, x2 = (x1 << 8) | c1;
    x = p2 ? x2 : (p1 ? x1 : xn);
    pos += __popc(b1) + __popc(b2);
  }
  return s;
}

// nfull full rounds in slot-table mode from a round boundary (st.next a
// multiple of 32), handing each round's symbol to emit(s) in order.  The ring
// is checked once per U rounds (U = 2 or 4): a round reads at most 64 bytes,
// so U rounds after a check, which leaves the position less than one segment
// into the ring, stay inside its first 1 + U / 2 segments; the check lets at
// most RING / 128 - 1 - U / 2 segment fills stay in flight, and runs once
// more at the end.
template <uint32_t RING = kRing, uint32_t U = 2, class Emit>
__device__ __forceinline__ void table_full_rounds(Stream& st, uint8_t* ring, const Lut& lut, uint32_t nfull,
                                                  uint32_t lane, uint32_t lt, Emit&& emit) {
  static_assert(U == 2 || U == 4, "two or four rounds per ring check");
  uint32_t x = st.x, pos = st.pos, base = st.base;
  auto check = [&]() {
    while (pos >= base + kSeg) {
      ring_issue<RING>(st, ring, base + RING, lane);
      base += kSeg;
      cp_async_wait<RING / kSeg - 1 - U / 2>();
      __syncwarp();
    }
  };
  uint32_t r = 0;
  for (; r + U <= nfull; r += U) {
    check();
#pragma unroll
    for (uint32_t u = 0; u < U; u++) emit(table_round<RING>(x, pos, ring, lut, lt));
  }
  for (; r < nfull; r++) {
    check();
    emit(table_round<RING>(x, pos, ring, lut, lt));
  }
  check();  // the single-round decoders that follow expect less than one segment consumed
  st.x = x;
  st.pos = pos;
  st.base = base;
  st.next += 32 * nfull;
}

// All symbols consumed, all bytes consumed and every state back at L.
__device__ __forceinline__ bool stream_finished(const Stream& st) {
  bool ok = st.next == st.nsym && st.pos == st.nbytes && (st.nsym == 0 || st.x == ACE_RANS_L);
  return __all_sync(kFull, ok);
}

}  // namespace ace
