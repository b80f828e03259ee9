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
  uint32_t pad[52];
};
static_assert(sizeof(ScratchHdr) == 256, "scratch header");

// First 256 bytes of the index memory.
struct IndexHdr {
  uint32_t status;
  uint32_t err_block;
  uint32_t err_where;
  uint32_t n_levels;
  uint32_t pad[60];
};
static_assert(sizeof(IndexHdr) == 256, "index header");

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

__device__ __forceinline__ uint32_t ld_acquire(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_release(uint32_t* p, uint32_t v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Spins until *flag == want or timeout_ns passes; false on timeout.
__device__ __forceinline__ bool wait_flag(const uint32_t* flag, uint32_t want, uint64_t timeout_ns) {
  if (ld_acquire(flag) == want) return true;
  uint64_t t0 = globaltimer();
  uint32_t ns = 32;
  while (true) {
    __nanosleep(ns);
    if (ld_acquire(flag) == want) return true;
    if (globaltimer() - t0 > timeout_ns) return false;
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

// State of one interleaved-rANS stream being decoded by a warp: lane j holds
// the state of interleaved lane j; pos/next are warp-uniform.
struct Rans {
  const uint8_t* bytes;  // renormalisation bytes (global)
  uint32_t nbytes;       // their count
  uint32_t pos;          // bytes consumed
  uint32_t next;         // next symbol index to decode
  uint32_t nsym;
  uint32_t x;            // this lane's state
};

// Reads one stream's entry states and frequency table and builds its lookup
// tables (the entropy layer's per-block entry point, Section 3).  The stream
// bounds were validated when the index was built.  Returns false (all lanes)
// on a bad table or state.
__device__ __forceinline__ bool stream_setup(const uint8_t* sp, uint32_t sbytes, uint32_t nsym, Lut& lut,
                                             Rans& r, uint32_t lane) {
  r.nsym = nsym;
  r.next = 0;
  r.pos = 0;
  r.x = ACE_RANS_L;
  r.bytes = sp;
  r.nbytes = 0;
  if (nsym == 0) return sbytes == 0;
  uint32_t x = reinterpret_cast<const uint32_t*>(sp)[lane];
  bool bad = x < ACE_RANS_L || x >= (1u << 31);
  uint32_t bm = sp[128 + lane];
  uint32_t cnt = __popc(bm);
  uint32_t incl = warp_incl_sum(cnt, lane);
  uint32_t first = incl - cnt;
  uint32_t present = __shfl_sync(kFull, incl, 31);
  uint32_t head = ACE_STREAM_HEAD + ((2 * present + 15) & ~15u);
  bad |= head > sbytes;
  uint32_t f[8], fsum = 0;
  const uint8_t* fp = sp + ACE_STREAM_HEAD;
  uint32_t k = first;
#pragma unroll
  for (int j = 0; j < 8; j++) {
    f[j] = 0;
    if ((bm >> j) & 1) {
      if (!bad) f[j] = (uint32_t)fp[2 * k] | ((uint32_t)fp[2 * k + 1] << 8);
      k++;
      bad |= f[j] == 0 || f[j] > ACE_SCALE;
    }
    fsum += f[j];
  }
  uint32_t cincl = warp_incl_sum(fsum, lane);
  bad |= __shfl_sync(kFull, cincl, 31) != ACE_SCALE;
  if (__any_sync(kFull, bad)) return false;
  // slot -> symbol: zero the table, mark each symbol's first slot, prefix-max
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
  r.bytes = sp + head;
  r.nbytes = sbytes - head;
  r.x = x;
  return true;
}

// Decodes symbols [r.next, end) of a stream; symbol i is on lane i mod 32.
// sink(i, s) receives each symbol on the lane that decoded it.  Renormalisation
// bytes are taken in symbol order: a lane needing k in {0,1,2} bytes reads
// them at the running position plus the bytes needed by lower lanes, high
// byte first.  Returns false (all lanes) if the stream runs out of bytes.
template <class Sink>
__device__ __forceinline__ bool rans_decode(Rans& r, const Lut& lut, uint32_t end, uint32_t lane, Sink&& sink) {
  const uint32_t lt = lanemask_lt();
  while (r.next < end) {
    uint32_t base = r.next & ~31u;
    uint32_t i = base + lane;
    bool act = i >= r.next && i < end;
    uint32_t x = r.x, k = 0, s = 0;
    if (act) {
      uint32_t slot = x & (ACE_SCALE - 1);
      s = lut.sym[slot];
      uint32_t fc = lut.fc[s];
      x = (fc >> 16) * (x >> ACE_SCALE_BITS) + slot - (fc & 0xffffu);
      k = (x < (1u << 15)) + (x < ACE_RANS_L);
    }
    uint32_t b1 = __ballot_sync(kFull, k >= 1), b2 = __ballot_sync(kFull, k == 2);
    uint32_t pre = __popc(b1 & lt) + __popc(b2 & lt);
    uint32_t tot = __popc(b1) + __popc(b2);
    if (r.pos + tot > r.nbytes) return false;
    const uint8_t* p = r.bytes + r.pos + pre;
    if (k >= 1) x = (x << 8) | p[0];
    if (k == 2) x = (x << 8) | p[1];
    r.pos += tot;
    if (act) {
      r.x = x;
      sink(i, s);
    }
    r.next = min(base + 32, end);
  }
  return true;
}

// All symbols consumed, all bytes consumed and every state back at L.
__device__ __forceinline__ bool rans_finished(const Rans& r) {
  bool ok = r.next == r.nsym && r.pos == r.nbytes && (r.nsym == 0 || r.x == ACE_RANS_L);
  return __all_sync(kFull, ok);
}

}  // namespace ace
