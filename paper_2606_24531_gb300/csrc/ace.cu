// GPU library of the two-layer codec: block index, fused two-layer decode
// (whole archive and unified seek), closure search, verification, and the
// C ABI declared in include/ace.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "ace.h"
#include "ace_device.cuh"
#include "ace_format.h"

using namespace ace;

namespace {

constexpr uint64_t kDefaultTimeoutNs = 2000000000ull;
constexpr uint32_t kMaxLevelLaunches = 32;  // whole decodes with more levels wait on flags instead
// A seek's closure marks its blocks' ready flags with the call's epoch and
// this bit; publishing a decoded block clears it.  A source block whose flag
// shows neither is outside the closure: the archive is corrupt.  (Epochs
// count calls on one scratch buffer and stay below 2^31.)
constexpr uint32_t kPendingFlag = 0x80000000u;

inline uint64_t align256(uint64_t v) { return (v + 255) & ~255ull; }

__host__ __device__ inline uint32_t esc_cap(uint32_t log2B) { return 2 * ((1u << log2B) / 255) + 2; }

// ------------------------------------------------------------ index kernels

struct IndexArgs {
  uint64_t* match_ptr;  // n_blocks + 1 entries: first match record of each block
  const uint8_t* arc;
  const ace_block_dir* dir;
  const uint32_t* dep_ptr;
  const uint32_t* dep_iv;
  IndexHdr* ih;
  uint32_t* level;
  uint32_t* order;
  uint32_t* lv_count;  // n_blocks + 1 entries
  uint32_t* lv_cursor; // n_blocks + 1 entries
  uint64_t nb, total, payload_off, arc_bytes, deps_off;
  uint64_t max_iv;  // intervals that fit between the pointer table and the payload
  uint32_t log2B, w;
};

// Checks every directory entry and dependency record so the decoder may trust
// stream bounds and token counts (Section 2 block layout, Section 3 streams).
__global__ void validate_kernel(IndexArgs a) {
  uint64_t b = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (b == 0) {  // the interval table must end before the payload
    const uint32_t niv = a.dep_ptr[a.nb];
    a.ih->n_iv = niv;
    if (a.deps_off + 4 * (a.nb + 1) + 8ull * niv > a.payload_off)
      record_error(&a.ih->status, &a.ih->err_block, &a.ih->err_where, ACE_E_CORRUPT, 0, 12);
  }
  if (b >= a.nb) return;
  const ace_block_dir d = a.dir[b];
  uint64_t B = (uint64_t)1 << a.log2B, bstart = b << a.log2B;
  uint64_t blen = min(B, a.total - bstart);
  uint32_t where = 0;
  for (int k = 0; k < 3 && !where; k++) {
    if (d.mode[k] > 1) where = 1;  // 0: rANS, 1: stored
    else if (d.nsym[k] == 0 && d.stream_bytes[k] != 0) where = 2;
    else if (d.nsym[k] != 0) {
      if (d.mode[k] == 1 ? d.stream_bytes[k] != d.nsym[k] : d.stream_bytes[k] < ACE_STREAM_HEAD) where = 3;
      else if (d.stream_off[k] & 15) where = 3;
      else if (a.payload_off + d.stream_off[k] + d.stream_bytes[k] > a.arc_bytes ||
               d.stream_off[k] > a.arc_bytes)
        where = 4;
    }
  }
  if (!where) {
    if (d.ntok == 0 || d.ntok > blen + 1) where = 5;
    else if (d.nsym[ACE_S_LIT] > blen) where = 6;
    else if ((uint64_t)d.nsym[ACE_S_LEN] != 2ull * d.nesc + 2ull * d.ntok) where = 7;
    else if ((uint64_t)d.nsym[ACE_S_OFF] != (uint64_t)a.w * (d.ntok - 1)) where = 8;
    else if (d.nesc > esc_cap(a.log2B)) where = 9;
  }
  if (!where) {
    uint32_t lo = a.dep_ptr[b], hi = a.dep_ptr[b + 1], niv = a.dep_ptr[a.nb];
    if (lo > hi || hi > niv || hi > a.max_iv) where = 10;  // intervals read below stay before the payload
    else
      for (uint32_t i = lo; i < hi && !where; i++) {
        uint32_t f = a.dep_iv[2 * i], l = a.dep_iv[2 * i + 1];
        if (f > l || l >= b) where = 11;
      }
  }
  if (where) record_error(&a.ih->status, &a.ih->err_block, &a.ih->err_where, ACE_E_CORRUPT, (uint32_t)b, where);
  else atomicMax(&a.ih->max_ntok, d.ntok);
  a.match_ptr[b + 1] = d.ntok ? d.ntok - 1 : 0;  // this block's matches; scanned below
}

// Inclusive scan of the per-block match counts into record offsets (one CTA).
__global__ void match_scan_kernel(IndexArgs a) {
  __shared__ unsigned long long carry;
  __shared__ unsigned long long wsum[32];
  if (threadIdx.x == 0) {
    carry = 0;
    a.match_ptr[0] = 0;
  }
  __syncthreads();
  uint32_t lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (uint64_t c0 = 1; c0 <= a.nb; c0 += blockDim.x) {
    uint64_t i = c0 + threadIdx.x;
    unsigned long long v = i <= a.nb ? a.match_ptr[i] : 0, incl = v;
    for (int d = 1; d < 32; d <<= 1) {
      unsigned long long u = __shfl_up_sync(kFull, incl, d);
      if (lane >= (uint32_t)d) incl += u;
    }
    if (lane == 31) wsum[wid] = incl;
    __syncthreads();
    if (wid == 0) {
      unsigned long long x = lane < nw ? wsum[lane] : 0, xi = x;
      for (int d = 1; d < 32; d <<= 1) {
        unsigned long long u = __shfl_up_sync(kFull, xi, d);
        if (lane >= (uint32_t)d) xi += u;
      }
      if (lane < nw) wsum[lane] = xi - x;
    }
    __syncthreads();
    unsigned long long out = carry + wsum[wid] + incl;
    if (i <= a.nb) a.match_ptr[i] = out;
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) carry = out;
    __syncthreads();
  }
  if (threadIdx.x == 0) a.ih->n_matches = carry;
}

// Dependency levels: level[b] = 0 without sources in other blocks, else
// 1 + the deepest block it reads (Section 2).  Sources always precede, so
// one CTA walks the blocks in chunks and relaxes each chunk to its fixed point.
// One sweep of the dependency levels (Section 2: a block decodes once the
// blocks it reads are present), a warp per block with its lanes over the
// block's dependency intervals: level[b] <- max(level[b], 1 + the largest
// level of a block it reads).  Levels only grow toward each block's depth in
// the dependency graph, and reach it after as many sweeps as there are
// levels; a sweep that changes a level sets its flag.
constexpr uint32_t kLevelSweeps = 8;

__global__ void levels_sweep_kernel(IndexArgs a, uint32_t sweep) {
  __shared__ uint32_t changed;
  if (*(volatile uint32_t*)&a.ih->status) return;
  if (sweep > 0 && !*(volatile uint32_t*)&a.ih->relax[sweep - 1]) return;  // settled already
  if (threadIdx.x == 0) changed = 0;
  __syncthreads();
  const uint32_t lane = threadIdx.x & 31;
  const uint64_t nw = (uint64_t)gridDim.x * (blockDim.x >> 5);
  for (uint64_t b = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5; b < a.nb; b += nw) {
    uint32_t lv = 0;
    const uint32_t e1 = a.dep_ptr[b + 1];
    for (uint32_t e = a.dep_ptr[b] + lane; e < e1; e += 32)
      for (uint32_t k = a.dep_iv[2 * e]; k <= a.dep_iv[2 * e + 1]; k++) lv = max(lv, a.level[k] + 1);
#pragma unroll
    for (int d = 16; d; d >>= 1) lv = max(lv, __shfl_xor_sync(kFull, lv, d));
    if (lane == 0 && lv > a.level[b]) {
      a.level[b] = lv;
      changed = 1;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0 && changed) a.ih->relax[sweep] = 1;  // one store per CTA, not per block
}

// The levels in one CTA, block chunk by block chunk, for archives whose
// levels did not settle within the sweeps (deep dependency chains).
__global__ void levels_kernel(IndexArgs a) {
  __shared__ int changed;
  if (*(volatile uint32_t*)&a.ih->status || !*(volatile uint32_t*)&a.ih->relax[kLevelSweeps - 1]) return;
  for (uint64_t c0 = 0; c0 < a.nb; c0 += blockDim.x) {
    uint64_t b = c0 + threadIdx.x;
    if (b < a.nb) a.level[b] = 0;
    __syncthreads();
    while (true) {
      if (threadIdx.x == 0) changed = 0;
      __syncthreads();
      if (b < a.nb) {
        uint32_t lv = 0;
        for (uint32_t i = a.dep_ptr[b]; i < a.dep_ptr[b + 1]; i++)
          for (uint32_t k = a.dep_iv[2 * i]; k <= a.dep_iv[2 * i + 1]; k++) lv = max(lv, a.level[k] + 1);
        if (lv != a.level[b]) {
          a.level[b] = lv;
          changed = 1;
        }
      }
      __syncthreads();
      if (!changed) break;
      __syncthreads();
    }
  }
}

__global__ void level_hist_kernel(IndexArgs a) {
  if (*(volatile uint32_t*)&a.ih->status) return;
  uint64_t b = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (b < a.nb) {
    const uint32_t lv = a.level[b];
    atomicAdd(&a.lv_count[lv], 1u);
    atomicMax(&a.ih->n_levels, lv + 1);
  }
}

// Exclusive scan of the level histogram into level start offsets (one CTA).
__global__ void level_scan_kernel(IndexArgs a) {
  __shared__ uint32_t carry;
  __shared__ uint32_t wsum[32];
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  uint32_t lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (uint64_t c0 = 0; c0 < a.nb + 1; c0 += blockDim.x) {
    uint64_t i = c0 + threadIdx.x;
    uint32_t v = i < a.nb + 1 ? a.lv_count[i] : 0;
    uint32_t incl = warp_incl_sum(v, lane);
    if (lane == 31) wsum[wid] = incl;
    __syncthreads();
    if (wid == 0) {
      uint32_t s = lane < nw ? wsum[lane] : 0;
      uint32_t si = warp_incl_sum(s, lane);
      if (lane < nw) wsum[lane] = si - s;
    }
    __syncthreads();
    uint32_t ex = carry + wsum[wid] + incl - v;
    if (i < a.nb + 1) a.lv_cursor[i] = ex;
    if (i < 33) a.ih->lvc[i] = v;  // the host reads the first levels' sizes with the header
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) carry = ex + v;
    __syncthreads();
  }
}

__global__ void level_scatter_kernel(IndexArgs a) {
  if (*(volatile uint32_t*)&a.ih->status) return;
  uint64_t b = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (b < a.nb) a.order[atomicAdd(&a.lv_cursor[a.level[b]], 1u)] = (uint32_t)b;
}

// An index read back from storage, checked against its archive instead of
// rebuilt.  Each block's level must be the fixed point of the level rule
// (0 without dependencies, else 1 + the deepest block it reads): one sweep
// verifies what the build reaches by iterating.  A warp per block.
__global__ void level_verify_kernel(IndexArgs a) {
  if (*(volatile uint32_t*)&a.ih->status) return;
  const uint32_t lane = threadIdx.x & 31;
  const uint64_t nw = (uint64_t)gridDim.x * (blockDim.x >> 5);
  for (uint64_t b = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5; b < a.nb; b += nw) {
    uint32_t lv = 0;
    const uint32_t e1 = a.dep_ptr[b + 1];
    for (uint32_t e = a.dep_ptr[b] + lane; e < e1; e += 32)
      for (uint32_t k = a.dep_iv[2 * e]; k <= a.dep_iv[2 * e + 1]; k++) lv = max(lv, a.level[k] + 1);
#pragma unroll
    for (int d = 16; d; d >>= 1) lv = max(lv, __shfl_xor_sync(kFull, lv, d));
    if (lane == 0 && (lv != a.level[b] || lv >= a.ih->n_levels))
      record_error(&a.ih->status, &a.ih->err_block, &a.ih->err_where, ACE_E_CORRUPT, (uint32_t)b, 60);
  }
}

// The decode order of a stored index: a permutation of the blocks (seen
// marks each once), in non-decreasing level, position i inside its level's
// range of the order (the level's end in lv_cursor, its size in lv_count).
__global__ void order_verify_kernel(IndexArgs a, uint32_t* seen) {
  if (*(volatile uint32_t*)&a.ih->status) return;
  const uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  // the first levels' sizes in the header (the host's level ranges) match
  if (i < 33 && i < a.ih->n_levels && i <= a.nb && a.ih->lvc[i] != a.lv_count[i])
    record_error(&a.ih->status, &a.ih->err_block, &a.ih->err_where, ACE_E_CORRUPT, (uint32_t)i, 62);
  if (i >= a.nb) return;
  const uint32_t b = a.order[i];
  bool bad = b >= a.nb;
  if (!bad) {
    bad = atomicExch(seen + b, 1u) != 0;
    const uint32_t L = a.level[b];
    bad |= L >= a.ih->n_levels || L > a.nb;
    if (!bad) {
      const uint32_t end = a.lv_cursor[L], cnt = a.lv_count[L];
      bad |= i >= end || end < cnt || i < end - cnt;
    }
  }
  if (bad) record_error(&a.ih->status, &a.ih->err_block, &a.ih->err_where, ACE_E_CORRUPT, (uint32_t)i, 61);
}

// ----------------------------------------------------------- decode kernel

struct DecodeArgs {
  const uint8_t* arc;
  const ace_block_dir* dir;
  uint64_t payload_off;
  uint64_t total;
  uint64_t nb;
  uint32_t log2B, w;
  uint32_t window;         // tokens whose positions sit in shared memory at a time (multiple of 32)
  uint32_t esc_cap;        // escape values a block may hold
  uint32_t warp_smem;      // bytes of shared memory per warp
  uint32_t max_ntok;       // most tokens in any block
  uint32_t n_items;        // whole decode: work items; seek: read from the scratch header
  const uint32_t* items;   // whole decode: blocks in (level, block) order; seek: the closure
  uint8_t* out;            // whole decode: output (absolute positions); seek: block slots
  ScratchHdr* sh;
  uint32_t* ready;         // per block: the epoch once the block is decoded
  const uint32_t* slot_of; // seek: block -> slot
  uint32_t n_slots;        // seek: slots in the call's scratch (every slot_of entry read is checked against it)
  uint8_t* slice;          // seek: caller's output
  uint64_t coord, len;     // seek: requested range
  uint64_t timeout_ns;
  MatchRec* recs;          // match records, from the token pass to the literal and match passes
  const uint64_t* match_ptr;  // whole decode: block -> first record; null: max_ntok records per slot
  const uint32_t* level;   // each block's dependency level
  uint32_t cur_level;      // whole decode by levels: the level this launch resolves
  bool closure_flags;      // seek: the closure marked its blocks' ready flags (kPendingFlag)
  // fused schedule: per level the blocks whose matches are resolved, and
  // (whole decodes) the blocks the level holds (seeks read them from the
  // scratch header)
  uint32_t* lv_done;
  const uint32_t* lv_count;
  // seek batches: match records per work item rather than per slot
  const uint32_t* rec_index;
  uint32_t n_rec_slots;
  uint32_t long_min;       // matches at least this long (not overlapping) copy in 16-byte pieces
};

// Shared memory of one warp in the token pass: one stream's tables at a
// time, the length and offset streams' renormalisation rings, and the block's
// escape values.
struct TokMem {
  Lut* lut;
  uint8_t* ring;   // [2][kRing]: lengths, offsets
  uint16_t* esc;   // [esc_cap]
};

// Shared memory of one warp in the literal pass: the literal stream's tables
// and ring, and a window of token positions.
struct LitMem {
  Lut* lut;
  uint8_t* ring;   // [kRing]
  uint32_t* tdst;  // [window + 1] start of each token's literal run, within the block
  uint32_t* tlit;  // [window + 1] index of each token's first literal among the block's literals
};

constexpr uint32_t kMatchGroup = 32;  // matches whose records sit in shared memory at a time
// Groups of match records in flight to shared memory (a ring after the
// group's arrays of sources, destinations, lengths and copy starts).
constexpr uint32_t kRecDepth = 4;
constexpr uint32_t kRecRingOff = 20 * kMatchGroup + 16;
// The match pass keeps only its match-record area in shared memory.
constexpr uint32_t kMatchSmem = kRecRingOff + 16 * kMatchGroup * kRecDepth;

__host__ __device__ inline uint32_t tok_smem_bytes(uint32_t escn) {
  return (sizeof(Lut) + 2 * kRing + 2 * escn + 15) & ~15u;
}

// A plain seek's literal pass runs a handful of warps, each on its own
// critical path: a deeper ring keeps its renormalisation bytes ahead of it.
constexpr uint32_t kSeekRing = 2048;

__host__ __device__ inline uint32_t lit_smem_bytes(uint32_t window, uint32_t ring) {
  return (sizeof(Lut) + ring + 8 * (window + 1) + 15) & ~15u;
}

__device__ inline TokMem carve_tok(uint8_t* base) {
  TokMem m;
  m.lut = reinterpret_cast<Lut*>(base);
  m.ring = base + sizeof(Lut);
  m.esc = reinterpret_cast<uint16_t*>(m.ring + 2 * kRing);
  return m;
}

__device__ inline LitMem carve_lit(uint8_t* base, uint32_t window, uint32_t ring) {
  LitMem m;
  m.lut = reinterpret_cast<Lut*>(base);
  m.ring = base + sizeof(Lut);
  m.tdst = reinterpret_cast<uint32_t*>(m.ring + ring);
  m.tlit = m.tdst + (window + 1);
  return m;
}

// Slot of block k in a seek's scratch.  The entry is read back from scratch
// that earlier calls may have left in another state, so it is clamped to the
// call's slots: whatever it holds, the address stays inside the scratch (a
// block outside the call's closure is rejected before its bytes are used).
__device__ __forceinline__ uint32_t slot_index(const DecodeArgs& a, uint64_t k) {
  const uint32_t s = __ldg(a.slot_of + k);
  return s < a.n_slots ? s : 0u;
}
__device__ __forceinline__ uint64_t slot_base(const DecodeArgs& a, uint64_t k) {
  return (uint64_t)slot_index(a, k) << a.log2B;
}

template <bool SEEK>
struct Addr {
  // device address of absolute output position p
  __device__ __forceinline__ static const uint8_t* at(const DecodeArgs& a, uint64_t p) {
    if (SEEK) return a.out + slot_base(a, p >> a.log2B) + (p & ((1ull << a.log2B) - 1));
    return a.out + p;
  }
  // the same, with block b's own bytes at obase without a slot lookup
  __device__ __forceinline__ static const uint8_t* at(const DecodeArgs& a, uint64_t p, uint64_t b, const uint8_t* obase) {
    if (SEEK) {
      uint64_t k = p >> a.log2B;
      const uint64_t off = p & ((1ull << a.log2B) - 1);
      if (k == b) return obase + off;
      return a.out + slot_base(a, k) + off;
    }
    return a.out + p;
  }
};

__device__ __forceinline__ void fail(const DecodeArgs& a, bool& ok, ace_status code, uint32_t b, uint32_t where,
                                     uint32_t lane) {
  if (ok && lane == 0) record_error(&a.sh->status, &a.sh->err_block, &a.sh->err_where, code, b, where);
  ok = false;
}

// Source byte i of a match (sequential LZ77 semantics): with distance
// d = D - S, byte i of the destination equals byte S + (i mod d) when the
// source overlaps the destination (d < len), and S + i otherwise; either way
// every byte read precedes D and is final when the copy starts.
__device__ __forceinline__ uint64_t src_index(uint64_t S, uint64_t d, uint32_t len, uint32_t i) {
  return d >= len ? S + i : S + (i % (uint32_t)d);
}

__device__ __forceinline__ uint64_t read_src(const uint8_t* q, uint32_t w) {
  uint64_t S = (uint64_t)q[0] | ((uint64_t)q[1] << 8) | ((uint64_t)q[2] << 16) | ((uint64_t)q[3] << 24);
  if (w == 5) S |= (uint64_t)q[4] << 32;
  return S;
}

// The records of block b: whole decodes by the index's prefix count of
// matches; seeks max_ntok per slot; seek batches max_ntok per work item
// (rec_index: block -> its place in the batch's work list).
template <bool SEEK>
__device__ __forceinline__ MatchRec* recs_of(const DecodeArgs& a, uint32_t b) {
  if (!SEEK) return a.recs + __ldg(a.match_ptr + b);
  if (a.rec_index) {
    uint32_t w = __ldg(a.rec_index + b);
    if (w >= a.n_rec_slots) w = 0;  // the closure wrote it this batch; clamped all the same
    return a.recs + (uint64_t)w * a.max_ntok;
  }
  return a.recs + (uint64_t)slot_index(a, b) * a.max_ntok;
}

// n bytes from src to dst by one warp: 16-byte vectors, four per lane in
// flight, when both are 16-byte aligned, else sixteen independent byte loads
// per lane before their stores (a store may not be passed by a later load
// the compiler cannot prove disjoint, so each batch is written out whole).
__device__ __forceinline__ void warp_copy(uint8_t* dst, const uint8_t* src, uint64_t n, uint32_t lane) {
  if (((reinterpret_cast<uintptr_t>(dst) | reinterpret_cast<uintptr_t>(src)) & 15) == 0) {
    const uint64_t nv = n >> 4;
    const uint4* s4 = reinterpret_cast<const uint4*>(src);
    uint4* d4 = reinterpret_cast<uint4*>(dst);
    for (uint64_t v0 = 0; v0 < nv; v0 += 128) {
      uint4 t[4];
#pragma unroll
      for (uint32_t u = 0; u < 4; u++) {
        const uint64_t v = v0 + 32 * u + lane;
        if (v < nv) t[u] = __ldcg(s4 + v);
      }
#pragma unroll
      for (uint32_t u = 0; u < 4; u++) {
        const uint64_t v = v0 + 32 * u + lane;
        if (v < nv) d4[v] = t[u];
      }
    }
    for (uint64_t p = (nv << 4) + lane; p < n; p += 32) dst[p] = __ldcg(src + p);
    return;
  }
  for (uint64_t p0 = 0; p0 < n; p0 += 512) {
    uint8_t t[16];
#pragma unroll
    for (uint32_t u = 0; u < 16; u++) {
      const uint64_t p = p0 + 32 * u + lane;
      if (p < n) t[u] = __ldcg(src + p);
    }
#pragma unroll
    for (uint32_t u = 0; u < 16; u++) {
      const uint64_t p = p0 + 32 * u + lane;
      if (p < n) dst[p] = t[u];
    }
  }
}

// Token pass of one block (Section 3: the block boundary is the entry point
// of the entropy layer): the length stream parsed into token positions, the
// offset stream, and one record per match -- absolute source, destination in
// the block, length -- for the match pass; the literal pass rebuilds the
// token positions from these records.  Returns false if the block is corrupt
// (the error is recorded).
template <bool SEEK>
__device__ bool token_block(const DecodeArgs& a, const TokMem& m, uint32_t b, uint32_t lane) {
  bool ok = true;
  const uint32_t* dw = reinterpret_cast<const uint32_t*>(a.dir + b);
  uint32_t dv = lane < 16 ? __ldg(dw + lane) : 0u;
  const uint64_t B = (uint64_t)1 << a.log2B, bstart = (uint64_t)b << a.log2B;
  const uint32_t blen = (uint32_t)min(B, a.total - bstart);
  const uint32_t w = a.w;
  const uint32_t ntok = __shfl_sync(kFull, dv, 12), nesc = __shfl_sync(kFull, dv, 13);
  const uint32_t nlit = __shfl_sync(kFull, dv, 9 + ACE_S_LIT);
  const uint32_t modes = __shfl_sync(kFull, dv, 14);  // mode[k] in byte k
  const uint32_t lt = lanemask_lt();

  Stream sn, so;
#pragma unroll
  for (int k = ACE_S_LEN; k <= ACE_S_OFF; k++) {
    uint64_t soff = (uint64_t)__shfl_sync(kFull, dv, 2 * k) | ((uint64_t)__shfl_sync(kFull, dv, 2 * k + 1) << 32);
    uint32_t sbytes = __shfl_sync(kFull, dv, 6 + k), nsym = __shfl_sync(kFull, dv, 9 + k);
    if (!stream_open(a.arc + a.payload_off + soff, sbytes, nsym, m.ring + (k - ACE_S_LEN) * kRing,
                     k == ACE_S_LEN ? sn : so, lane, (modes >> (8 * k)) & 0xffu))
      fail(a, ok, ACE_E_CORRUPT, b, 20 + k, lane);
  }
  if (!ok || ntok > a.max_ntok) {
    fail(a, ok, ACE_E_CORRUPT, b, 23, lane);
    cp_async_wait<0>();
    __syncwarp();
    return false;
  }
  cp_async_wait<2>();
  __syncwarp();
  uint8_t* rn = m.ring;
  uint8_t* ro = m.ring + kRing;

  // ---- lengths: escape values, then two codes per token
  if (!lut_build(sn, *m.lut, lane)) fail(a, ok, ACE_E_CORRUPT, b, 30, lane);
  uint8_t* escb = reinterpret_cast<uint8_t*>(m.esc);
  if (ok)
    rans_run(sn, rn, *m.lut, 2 * nesc, lane, lt, [&](bool act, uint32_t i, uint32_t s) {
      if (act) escb[i] = (uint8_t)s;
    });
  __syncwarp();
  uint32_t out_pos = 0, lit_pos = 0, esc_rank = 0;
  bool bad = false;
  const uint32_t cbase = 2 * nesc, cend = cbase + 2 * ntok;
  // match t's record is written whole here (destination and length; the
  // source's bytes follow from the offset stream); a match ends token t
  // (t < ntok - 1), its destination is the token's start plus its run
  uint4* const rec4 = reinterpret_cast<uint4*>(recs_of<SEEK>(a, b));
  if (ok) rans_run(sn, rn, *m.lut, cend, lane, lt, [&](bool act, uint32_t i, uint32_t s) {
    bool e = act && s == 255;
    uint32_t eb = __ballot_sync(kFull, e);
    uint32_t r = esc_rank + __popc(eb & lt);
    uint32_t v = s;
    if (e) {
      if (r < nesc) v = 255u + m.esc[r];
      else bad = true;
    }
    esc_rank += __popc(eb);
    uint32_t lr = __shfl_sync(kFull, v, lane & ~1u), ml = __shfl_sync(kFull, v, lane | 1u);
    bool own = act && !(lane & 1);  // codes start at an even index: pairs never straddle rounds
    uint32_t to = own ? lr + ml : 0u, tl = own ? lr : 0u;
    uint32_t io = warp_incl_sum(to, lane), il = warp_incl_sum(tl, lane);
    if (own) {
      uint32_t t = (i - cbase) >> 1;
      if (t + 1 < ntok) rec4[t] = make_uint4(0u, 0u, out_pos + io - to + lr, ml);
      else if (ml) bad = true;  // the block's last token carries no match
    }
    out_pos += __shfl_sync(kFull, io, 31);
    lit_pos += __shfl_sync(kFull, il, 31);
    if (out_pos > blen) bad = true;
  });
  bad |= out_pos != blen || lit_pos != nlit || esc_rank != nesc;
  if (__any_sync(kFull, bad)) fail(a, ok, ACE_E_CORRUPT, b, 32, lane);

  // ---- absolute offsets: off_width bytes for every token but the last
  const uint32_t nm = ntok - 1;
  if (ok && nm) {
    __syncwarp();  // the records' zero source bytes are written before any lane fills them
    if (!lut_build(so, *m.lut, lane)) fail(a, ok, ACE_E_CORRUPT, b, 33, lane);
    const uint32_t oend = w * nm;
    // offset byte i is byte i mod w of match i / w's absolute source (little
    // endian, w = 4 or 5), written straight into its record
    uint8_t* const rb = reinterpret_cast<uint8_t*>(rec4);
    auto at = [&](uint32_t i) -> uint8_t* {
      const uint32_t t = w == 4 ? i >> 2 : __umulhi(i, 0xCCCCCCCDu) >> 2;  // floor(i / 5) for every 32-bit i
      return rb + 16 * (size_t)t + (i - w * t);
    };
    auto put = [&](bool act, uint32_t i, uint32_t s) {
      if (act) *at(i) = (uint8_t)s;
    };
    if (ok && !so.stored && so.k == 0 && oend >= 64) {  // slot-table streams: full rounds in the fast loop
      uint32_t i = lane;
      table_full_rounds(so, ro, *m.lut, oend >> 5, lane, lt, [&](uint32_t s) {
        *at(i) = (uint8_t)s;
        i += 32;
      });
    }
    if (ok) rans_run(so, ro, *m.lut, oend, lane, lt, put);
  }
  __syncwarp();
  // a source at or after its destination is caught where sources are read:
  // match_block and match_small_kernel check every record
  if (ok) {
    bool fin = stream_finished(sn) && stream_finished(so);
    if (!__all_sync(kFull, fin)) fail(a, ok, ACE_E_CORRUPT, b, 40, lane);
  }
  cp_async_wait<0>();  // no ring fill may land after the next block reuses the rings
  __syncwarp();
  return ok;
}

// Literal pass of one block, after the token pass of every block succeeded:
// literal i lands at its token's run start plus its place in the run.  Token
// positions come into a shared-memory window from the match records: token
// t's run starts where the previous match ended and ends at its own match's
// destination (the last token's at the block end).  Returns false if the
// literal stream is corrupt.
template <bool SEEK, uint32_t RING>
__device__ bool literal_block(const DecodeArgs& a, const LitMem& m, uint32_t b, uint32_t lane) {
  bool ok = true;
  const uint32_t* dw = reinterpret_cast<const uint32_t*>(a.dir + b);
  uint32_t dv = lane < 16 ? __ldg(dw + lane) : 0u;
  const uint64_t B = (uint64_t)1 << a.log2B, bstart = (uint64_t)b << a.log2B;
  const uint32_t blen = (uint32_t)min(B, a.total - bstart);
  const uint32_t ntok = __shfl_sync(kFull, dv, 12);
  const uint32_t nm = ntok ? ntok - 1 : 0;
  uint8_t* obase = SEEK ? a.out + slot_base(a, b) : a.out + bstart;
  const uint32_t lt = lanemask_lt();
  Stream sl;
  {
    const int k = ACE_S_LIT;
    uint64_t soff = (uint64_t)__shfl_sync(kFull, dv, 2 * k) | ((uint64_t)__shfl_sync(kFull, dv, 2 * k + 1) << 32);
    uint32_t sbytes = __shfl_sync(kFull, dv, 6 + k), nsym = __shfl_sync(kFull, dv, 9 + k);
    const uint32_t mode = __shfl_sync(kFull, dv, 14) & 0xffu;
    if (!stream_open<RING>(a.arc + a.payload_off + soff, sbytes, nsym, m.ring, sl, lane, mode))
      fail(a, ok, ACE_E_CORRUPT, b, 20, lane);
  }
  cp_async_wait<RING / kSeg - 2>();
  __syncwarp();
  if (ok && sl.nsym) {
    if (!lut_build(sl, *m.lut, lane)) fail(a, ok, ACE_E_CORRUPT, b, 35, lane);
    const uint4* rec = reinterpret_cast<const uint4*>(recs_of<SEEK>(a, b));
    uint32_t cdst = 0, clit = 0;  // run start and first literal of the window's first token
    for (uint32_t w0 = 0; ok && w0 < ntok; w0 += a.window) {
      const uint32_t wn = min(a.window, ntok - w0);
      for (uint32_t k0 = 0; k0 < wn; k0 += 32) {
        const uint32_t k = k0 + lane, t = w0 + k;
        uint32_t D = blen, L = 0;  // the last token's run ends at the block end
        if (k < wn && t < nm) {
          const uint4 r = __ldcg(rec + t);
          D = r.z;
          L = r.w;
        }
        const uint32_t end = D + L;  // where the next token's run starts
        const uint32_t prev = __shfl_up_sync(kFull, end, 1);
        const uint32_t st0 = lane ? prev : cdst;
        const uint32_t lr = k < wn ? D - st0 : 0u;
        const uint32_t incl = warp_incl_sum(lr, lane);
        if (k < wn) {
          m.tdst[k] = st0;
          m.tlit[k] = clit + incl - lr;
        }
        const uint32_t last = min(31u, wn - 1 - k0);
        cdst = __shfl_sync(kFull, end, last);
        clit += __shfl_sync(kFull, incl, last);
      }
      if (lane == 0) {
        m.tdst[wn] = cdst;
        m.tlit[wn] = clit;
      }
      __syncwarp();
      const uint32_t lend = m.tlit[wn];
      if (lend > sl.nsym) {  // the token pass checked these counts: only a changed archive gets here
        fail(a, ok, ACE_E_CORRUPT, b, 36, lane);
        break;
      }
      uint32_t tp = 0, cur_lit = m.tlit[0], cur_dst = m.tdst[0], nxt_lit = m.tlit[1];
      auto place = [&](bool act, uint32_t i, uint32_t s) {
        if (act) {
          while (nxt_lit <= i) {
            tp++;
            cur_lit = nxt_lit;
            cur_dst = m.tdst[tp];
            nxt_lit = m.tlit[tp + 1];
          }
          obase[cur_dst + (i - cur_lit)] = (uint8_t)s;
        }
      };
      if (!sl.stored && sl.k == 0 && lend - sl.next >= 64) {
        // slot-table streams: a partial round up to a round boundary, then
        // full rounds, each lane's literal pointer moving 32 bytes a round
        // until its literal index passes into the next token's run
        if (sl.next & 31) {
          bool act;
          uint32_t i;
          const uint32_t s = rans_round<RING>(sl, m.ring, *m.lut, lend, lane, lt, act, i);
          place(act, i, s);
        }
        const uint32_t nfull = (lend - sl.next) >> 5;
        uint32_t i = sl.next + lane;
        auto seek_token = [&]() {
          while (nxt_lit <= i) {
            tp++;
            cur_lit = nxt_lit;
            cur_dst = m.tdst[tp];
            nxt_lit = m.tlit[tp + 1];
          }
          return obase + cur_dst + (i - cur_lit);
        };
        uint8_t* op = seek_token();
        table_full_rounds<RING, 4>(sl, m.ring, *m.lut, nfull, lane, lt, [&](uint32_t s) {
          if (i >= nxt_lit) op = seek_token();
          *op = (uint8_t)s;
          op += 32;
          i += 32;
        });
      }
      rans_run<RING>(sl, m.ring, *m.lut, lend, lane, lt, place);
      __syncwarp();
    }
  }
  if (ok) {
    bool fin = stream_finished(sl);
    if (!__all_sync(kFull, fin)) fail(a, ok, ACE_E_CORRUPT, b, 41, lane);
  }
  cp_async_wait<0>();
  __syncwarp();
  return ok;
}

// Matches per lane in a group: match j of the group is on lane j mod 32.
constexpr uint32_t kLaneMatches = kMatchGroup / 32;
// Bytes in flight per lane in the bytewise copy of a round's matches.
constexpr uint32_t kCopyUnroll = 8;
// 16-byte pieces in flight per lane in the copy of a round's long matches.
constexpr uint32_t kLongUnroll = 2;
// Copy classes: a non-overlapping match of at most kShortMax bytes is copied
// by one lane in aligned 8-byte words, one of at least the call's long_min
// bytes by the whole warp in aligned 16-byte pieces, every other one
// bytewise with the round's other such matches.  long_min is the copy-width
// knob: kLongMinWide (16-byte pieces for everything above the short class)
// or kLongMinNarrow (bytewise up to 511 bytes).
constexpr uint32_t kShortMax = 32;
constexpr uint32_t kLongMinNarrow = 512;
constexpr uint32_t kLongMinWide = kShortMax + 1;

// A load of match source bytes.  L1: through the SM's L1 cache, for a pass
// whose sources were all written by earlier launches or by this warp (one
// launch per dependency level); else at L2 only, which every SM sees
// coherently (source blocks published by other warps of the same launch).
template <bool L1, class T>
__device__ __forceinline__ T ld_src(const T* p) {
  return L1 ? __ldca(p) : __ldcg(p);
}

// Source of a short match: the aligned 8-byte words covering [S, S + len).
template <bool SEEK, bool L1>
__device__ __forceinline__ void short_load(const DecodeArgs& a, uint64_t S, uint32_t len, uint64_t (&w)[5], uint64_t b,
                                           const uint8_t* obase) {
  const uint64_t a0 = S & ~7ull;
  const uint32_t off = (uint32_t)(S & 7);
#pragma unroll
  for (uint32_t k = 0; k < 5; k++) {
    const uint64_t q = a0 + 8ull * k;
    w[k] = 0;
    if (8 * k < off + len) {
      if (q + 8 <= a.total) {
        w[k] = ld_src<L1>(reinterpret_cast<const unsigned long long*>(Addr<SEEK>::at(a, q, b, obase)));
      } else {
        for (uint32_t t = 0; t < 8 && q + t < a.total; t++)
          w[k] |= (uint64_t)ld_src<L1>(Addr<SEEK>::at(a, q + t, b, obase)) << (8 * t);
      }
    }
  }
}

// Bytes sh .. sh + 7 of hi:lo (sh < 8).
__device__ __forceinline__ uint64_t funnel64(uint64_t lo, uint64_t hi, uint32_t sh) {
  return sh ? (lo >> (8 * sh)) | (hi << (64 - 8 * sh)) : lo;
}

// Bytes [lo, hi) of w to the 8-byte aligned p, in the widest aligned stores
// that fit.  The lanes of a round store to different lines, so every store
// a lane saves is an L1 and L2 transaction saved.
__device__ __forceinline__ void store_bytes8(uint8_t* p, uint64_t w, uint32_t lo, uint32_t hi) {
  uint32_t k = lo;
  while (k < hi) {
    if (!(k & 3) && k + 4 <= hi) {
      *reinterpret_cast<uint32_t*>(p + k) = (uint32_t)(w >> (8 * k));
      k += 4;
    } else if (!(k & 1) && k + 2 <= hi) {
      *reinterpret_cast<uint16_t*>(p + k) = (uint16_t)(w >> (8 * k));
      k += 2;
    } else {
      p[k] = (uint8_t)(w >> (8 * k));
      k++;
    }
  }
}

// Destination of a short match: aligned 8-byte words where the match covers
// them, the widest aligned stores that fit at its two ends.  Source byte off + i (off = S mod 8,
// counted from the first source word) lands at dp[i].
__device__ __forceinline__ void short_store(uint8_t* dp, uint32_t off, uint32_t len, const uint64_t (&w)[5]) {
  const uint32_t hd = (uint32_t)(reinterpret_cast<uintptr_t>(dp) & 7);
  uint8_t* dal = dp - hd;
  const bool same = off >= hd;  // destination word i starts in source word i, else in word i - 1
  const uint32_t sh = (off - hd) & 7;
#pragma unroll
  for (uint32_t i = 0; i < 5; i++) {
    const int first = 8 * (int)i - (int)hd;  // match byte held by the word's first byte
    if (first >= (int)len) break;
    const uint64_t lo = same ? w[i] : (i ? w[i - 1] : 0ull);
    const uint64_t hi = same ? (i + 1 < 5 ? w[i + 1] : 0ull) : w[i];
    const uint64_t word = funnel64(lo, hi, sh);
    if (first >= 0 && first + 8 <= (int)len) {
      *reinterpret_cast<uint64_t*>(dal + 8 * i) = word;
    } else {
      store_bytes8(dal + 8 * i, word, (uint32_t)max(0, -first), (uint32_t)min(8, (int)len - first));
    }
  }
}

// The 16 bytes at absolute output position q (a multiple of 16, possibly
// negative), bytes outside [0, total) read as zero.  An aligned piece never
// straddles a block (blocks are multiples of 256 bytes), so a seek finds it
// in one slot.
template <bool SEEK, bool L1>
__device__ __forceinline__ uint4 ld16_abs(const DecodeArgs& a, int64_t q, uint64_t b, const uint8_t* obase) {
  if (q >= 0 && (uint64_t)q + 16 <= a.total)
    return ld_src<L1>(reinterpret_cast<const uint4*>(Addr<SEEK>::at(a, (uint64_t)q, b, obase)));
  uint4 v = make_uint4(0, 0, 0, 0);
#pragma unroll 1
  for (uint32_t k = 0; k < 16; k++) {
    const int64_t p = q + k;
    if (p < 0 || (uint64_t)p >= a.total) continue;
    const uint32_t x = (uint32_t)ld_src<L1>(Addr<SEEK>::at(a, (uint64_t)p, b, obase)) << (8 * (k & 3));
    if (k < 4) v.x |= x;
    else if (k < 8) v.y |= x;
    else if (k < 12) v.z |= x;
    else v.w |= x;
  }
  return v;
}

// Bytes [lo, hi) of v to the 16-byte aligned p, in the widest aligned
// stores that fit (a piece at either end of a match).
__device__ __forceinline__ void store_bytes16(uint8_t* p, uint4 v, uint32_t lo, uint32_t hi) {
  auto word = [&](uint32_t k) { return k < 4 ? v.x : k < 8 ? v.y : k < 12 ? v.z : v.w; };
  uint32_t k = lo;
  while (k < hi) {
    if (!(k & 7) && k + 8 <= hi) {
      *reinterpret_cast<uint2*>(p + k) = make_uint2(word(k), word(k + 4));
      k += 8;
    } else if (!(k & 3) && k + 4 <= hi) {
      *reinterpret_cast<uint32_t*>(p + k) = word(k);
      k += 4;
    } else if (!(k & 1) && k + 2 <= hi) {
      *reinterpret_cast<uint16_t*>(p + k) = (uint16_t)(word(k) >> (8 * (k & 3)));
      k += 2;
    } else {
      p[k] = (uint8_t)(word(k) >> (8 * (k & 3)));
      k++;
    }
  }
}

// Bytes r .. r + 15 of B:A (r < 16, the same on every lane).
__device__ __forceinline__ uint4 funnel128(uint4 A, uint4 B, uint32_t r) {
  const uint32_t t = 8 * (r & 3);
  uint32_t y0, y1, y2, y3, y4;
  switch (r >> 2) {
    case 0: y0 = A.x; y1 = A.y; y2 = A.z; y3 = A.w; y4 = B.x; break;
    case 1: y0 = A.y; y1 = A.z; y2 = A.w; y3 = B.x; y4 = B.y; break;
    case 2: y0 = A.z; y1 = A.w; y2 = B.x; y3 = B.y; y4 = B.z; break;
    default: y0 = A.w; y1 = B.x; y2 = B.y; y3 = B.z; y4 = B.w; break;
  }
  return make_uint4(__funnelshift_r(y0, y1, t), __funnelshift_r(y1, y2, t), __funnelshift_r(y2, y3, t),
                    __funnelshift_r(y3, y4, t));
}

__device__ __forceinline__ uint4 shfl_down16(uint4 v, uint32_t d) {
  return make_uint4(__shfl_down_sync(kFull, v.x, d), __shfl_down_sync(kFull, v.y, d), __shfl_down_sync(kFull, v.z, d),
                    __shfl_down_sync(kFull, v.w, d));
}


// Whether a bit of the 128-bit mask (P0, P1, P2, P3) is set in [lo, hi].
__device__ __forceinline__ bool any_in(uint32_t P0, uint32_t P1, uint32_t P2, uint32_t P3, uint32_t lo,
                                       uint32_t hi) {
  bool any = false;
#pragma unroll
  for (uint32_t w = 0; w < 4; w++) {
    const uint32_t P = w == 0 ? P0 : w == 1 ? P1 : w == 2 ? P2 : P3;
    const uint32_t wlo = 32 * w, whi = wlo + 31;
    if (lo > hi || hi < wlo || lo > whi) continue;
    uint32_t m = P;
    if (lo > wlo) m &= ~0u << (lo - wlo);
    if (hi < whi) m &= (2u << (hi - wlo)) - 1u;
    any |= m != 0;
  }
  return any;
}

// First index i in [0, n) with key(i) > x, for keys that never decrease.
template <class Key>
__device__ __forceinline__ uint32_t upper_bound(uint32_t n, uint32_t x, Key key) {
  uint32_t lo = 0, len = n;
  while (len) {
    const uint32_t h = len >> 1;
    if (key(lo + h) <= x) {
      lo += h + 1;
      len -= h + 1;
    } else {
      len = h;
    }
  }
  return lo;
}

// Match pass of one block (Section 2: a block decodes once the blocks holding
// its sources are present).  Groups of up to 32 matches: their records are
// loaded together; with WAIT the source blocks before this one are checked
// with overlapping relaxed loads (a bounded wait only for one not yet
// published); without it (one launch per dependency level) each source
// block's level must be below this launch's level, else the archive's
// dependency lists disagree with its matches.  Then the group resolves in
// rounds.  A match is ready in a round when no
// pending match of its block writes a byte its source reads; literal bytes
// are final after the literal pass.  The first pending match is always ready,
// so every round makes progress, and a round's ready matches read no byte
// another one writes.  Returns false if a record is corrupt or a wait gave up.
template <bool SEEK, bool WAIT, bool L1 = !WAIT>
__device__ bool match_block(const DecodeArgs& a, MatchRec* gm, uint32_t b, uint32_t lane, uint32_t epoch,
                            uint32_t nm, uint32_t lvl = 0) {
  // L1: every source was written before the launch or by this warp (one
  // launch per level), so source loads may go through L1; otherwise other
  // SMs wrote them during the launch and loads go to L2.  Without WAIT, lvl
  // is the block's level: its sources must lie in lower ones.
  constexpr bool kL1 = L1;
  bool ok = true, bad = false;
  const uint64_t B = (uint64_t)1 << a.log2B, bstart = (uint64_t)b << a.log2B;
  const uint32_t blen = (uint32_t)min(B, a.total - bstart);
  uint8_t* obase = SEEK ? a.out + slot_base(a, b) : a.out + bstart;
  const uint4* rec = reinterpret_cast<const uint4*>(recs_of<SEEK>(a, b));
  uint64_t* gS = reinterpret_cast<uint64_t*>(gm);                 // [kMatchGroup] sources
  uint32_t* gD = reinterpret_cast<uint32_t*>(gS + kMatchGroup);   // [kMatchGroup] destinations in the block
  uint32_t* gL = gD + kMatchGroup;                                // [kMatchGroup] lengths
  uint32_t* gX = gL + kMatchGroup;                                // [kMatchGroup + 1] starts in a round's copy
  // records reach a ring of kRecDepth groups by cp.async, kRecDepth - 1
  // groups ahead of the one resolving; lane j copies and later reads record
  // j of each group, so no lane reads another's copy
  uint4* const rring = reinterpret_cast<uint4*>(reinterpret_cast<uint8_t*>(gm) + kRecRingOff);
  auto issue = [&](uint32_t g) {  // one commit group per call, empty past the last record
    const uint32_t t = g * kMatchGroup;
#pragma unroll
    for (uint32_t q = 0; q < kLaneMatches; q++) {
      const uint32_t j = lane + 32 * q;
      if (t < nm && j < min(kMatchGroup, nm - t)) cp_async16(rring + (g % kRecDepth) * kMatchGroup + j, rec + t + j);
    }
    cp_async_commit();
  };
#pragma unroll
  for (uint32_t g = 0; g + 1 < kRecDepth; g++) issue(g);
  for (uint32_t t0 = 0, g = 0; ok && t0 < nm; t0 += kMatchGroup, g++) {
    const uint32_t gn = min(kMatchGroup, nm - t0);
    issue(g + kRecDepth - 1);
    cp_async_wait<kRecDepth - 1>();  // group g has landed
    uint4 r[kLaneMatches];
#pragma unroll
    for (uint32_t q = 0; q < kLaneMatches; q++) {
      const uint32_t j = lane + 32 * q;
      r[q] = j < gn ? rring[(g % kRecDepth) * kMatchGroup + j] : make_uint4(0, 0, 0, 0);
    }
    uint32_t pend = 0;
#pragma unroll
    for (uint32_t q = 0; q < kLaneMatches; q++) {
      const uint32_t j = lane + 32 * q;
      if (j >= gn) continue;
      const uint64_t S = (uint64_t)r[q].x | ((uint64_t)r[q].y << 32);
      uint32_t ml = r[q].w;
      if (ml && (S >= bstart + r[q].z || (uint64_t)r[q].z + ml > blen)) {  // checked again: the token pass may have failed
        bad = true;
        ml = 0;
      }
      gS[j] = S;
      gD[j] = r[q].z;
      gL[j] = ml;
      if (ml) pend |= 1u << q;
    }
    if (__any_sync(kFull, bad)) fail(a, ok, ACE_E_CORRUPT, b, 37, lane);
    if (!ok) break;
    __syncwarp();

    // source blocks before this one: all flags loaded, then compared
    uint32_t f0[kLaneMatches], f1[kLaneMatches], rng[kLaneMatches];
    uint32_t ext = 0;
#pragma unroll
    for (uint32_t q = 0; q < kLaneMatches; q++) {
      f0[q] = f1[q] = epoch;
      rng[q] = 1;  // lo = 1 > hi = 0: no match of the group feeds this one
      if (!(pend >> q & 1)) continue;
      const uint32_t j = lane + 32 * q;
      const uint64_t S = gS[j], D = bstart + gD[j];
      const uint64_t rend = S + min((uint64_t)gL[j], D - S);
      const uint64_t k0 = S >> a.log2B;
      if (k0 < b) {  // blocks k0 .. k1 hold the bytes before this block
        const uint64_t k1 = min((rend - 1) >> a.log2B, (uint64_t)b - 1);
        ext |= 1u << q;
        if (WAIT) {  // flags that other warps publish during the launch
          f0[q] = ld_relaxed(a.ready + k0);
          f1[q] = k1 != k0 ? ld_relaxed(a.ready + k1) : f0[q];
        } else {  // levels, fixed for the launch: through the read-only cache
          f0[q] = __ldg(a.level + k0);
          f1[q] = k1 != k0 ? __ldg(a.level + k1) : f0[q];
        }
      }
      if (rend > bstart) {  // bytes of this block: the group's matches writing them
        const uint32_t s_rel = S > bstart ? (uint32_t)(S - bstart) : 0u, e_rel = (uint32_t)(rend - bstart);
        const uint32_t lo = upper_bound(j, s_rel, [&](uint32_t i) { return gD[i] + gL[i]; });
        const uint32_t hi = upper_bound(j, e_rel - 1, [&](uint32_t i) { return gD[i]; });  // first with gD >= e_rel
        rng[q] = hi > lo ? (lo | ((hi - 1) << 8)) : 1u;
      }
    }
    if (WAIT) {
      bool timeout = false;
      // a source block must sit at a lower dependency level (work lists are
      // in level order, so it was handed out before this block and the wait
      // ends); the block cache keeps no levels and skips this check
      const uint32_t my_level = a.level ? __ldg(a.level + b) : 0u;
#pragma unroll
      for (uint32_t q = 0; q < kLaneMatches; q++) {
        if (!(ext >> q & 1)) continue;
        const uint32_t j = lane + 32 * q;
        const uint64_t S = gS[j], D = bstart + gD[j];
        const uint64_t rend = S + min((uint64_t)gL[j], D - S);
        const uint64_t k0 = S >> a.log2B, k1 = min((rend - 1) >> a.log2B, (uint64_t)b - 1);
        if (a.level) {
          bool low = true;
          for (uint64_t k = k0; k <= k1; k++) low &= __ldg(a.level + k) < my_level;
          if (!low) {
            bad = true;  // the dependency table disagrees with the matches
            continue;
          }
        }
        if (SEEK && a.closure_flags) {
          // every source block must be a member of this seek's closure: its
          // flag carries the call's epoch (pending or published).  Anything
          // else means the dependency table disagrees with the matches.
          bool member = (f0[q] & ~kPendingFlag) == epoch && (f1[q] & ~kPendingFlag) == epoch;
          for (uint64_t k = k0 + 1; member && k < k1; k++)
            member = (ld_relaxed(a.ready + k) & ~kPendingFlag) == epoch;
          if (!member) {
            bad = true;
            continue;
          }
        }
        if (f0[q] == epoch && f1[q] == epoch && k1 <= k0 + 1) continue;  // blocks between them: the bounded wait
        for (uint64_t k = k0; k <= k1 && !timeout; k++)
          if (!wait_flag(a.ready + k, epoch, a.timeout_ns, &a.sh->status)) timeout = true;
      }
      if (__any_sync(kFull, bad)) fail(a, ok, ACE_E_CORRUPT, b, 39, lane);
      if (__any_sync(kFull, timeout)) fail(a, ok, ACE_E_TIMEOUT, b, 38, lane);
      if (!ok) break;
      if (__any_sync(kFull, ext != 0)) fence_acquire();
      __syncwarp();  // any lane may copy a match whose flags another lane checked
    }
    // without WAIT the level check below need not hold up the copies: a
    // corrupt archive fails the call whatever bytes they wrote
    uint32_t chk = ext;

    while (__any_sync(kFull, pend != 0)) {
      // pending matches of the group, one bit each (words past the group's size are zero)
      const uint32_t P0 = __ballot_sync(kFull, pend & 1u);
      const uint32_t P1 = kLaneMatches > 1 ? __ballot_sync(kFull, pend & 2u) : 0u;
      const uint32_t P2 = kLaneMatches > 2 ? __ballot_sync(kFull, pend & 4u) : 0u;
      const uint32_t P3 = kLaneMatches > 3 ? __ballot_sync(kFull, pend & 8u) : 0u;
      uint32_t go = 0;
#pragma unroll
      for (uint32_t q = 0; q < kLaneMatches; q++)
        if ((pend >> q & 1) && !any_in(P0, P1, P2, P3, rng[q] & 0xffu, rng[q] >> 8)) go |= 1u << q;
      // classes: short (one lane), long (the warp), the rest bytewise
      uint32_t sgo = 0, lgo = 0;
#pragma unroll
      for (uint32_t q = 0; q < kLaneMatches; q++) {
        if (!(go >> q & 1)) continue;
        const uint32_t j = lane + 32 * q, ml = gL[j];
        if (bstart + gD[j] - gS[j] < ml) continue;  // overlapping: bytewise
        if (ml <= kShortMax) sgo |= 1u << q;
        else if (ml >= a.long_min) lgo |= 1u << q;
      }
      if (sgo) {  // short: the next match's loads go out before the previous one's stores
        uint64_t cur[5], nxt[5];
        uint32_t jc = lane + 32 * (__ffs(sgo) - 1), rest = sgo & (sgo - 1);
        short_load<SEEK, kL1>(a, gS[jc], gL[jc], cur, b, obase);
        while (true) {
          const uint32_t jn = rest ? lane + 32 * (__ffs(rest) - 1) : 0u;
          if (rest) short_load<SEEK, kL1>(a, gS[jn], gL[jn], nxt, b, obase);
          short_store(obase + gD[jc], (uint32_t)(gS[jc] & 7), gL[jc], cur);
          if (!rest) break;
          rest &= rest - 1;
          jc = jn;
#pragma unroll
          for (uint32_t k = 0; k < 5; k++) cur[k] = nxt[k];
        }
      }
      if (__any_sync(kFull, lgo != 0)) {
        // long: the round's long matches at once, laid end to end as the
        // aligned 16-byte source pieces each one needs (its destination
        // pieces plus one); piece c and piece c + 1 build destination piece
        // c.  A window gives lane l pieces c0 + 32 u + l, kLongUnroll in
        // flight; piece c + 1 is the next lane's, or for lane 31 the next
        // u's lane 0; the window's very last piece only serves as that
        // source, and the next window starts on it.  Each lane finds its
        // pieces' match by walking forward (pieces only grow).
        static_assert(kLaneMatches == 1, "one match per lane");
        const bool mine = lgo & 1;
        const uint32_t hd0 = gD[lane] & 15;  // block bases are 16-byte aligned
        const uint32_t np = mine ? ((hd0 + gL[lane] + 15) >> 4) + 1 : 0u;
        const uint32_t incl = warp_incl_sum(np, lane);
        gX[lane] = incl - np;
        if (lane == 31) gX[32] = incl;
        const uint32_t T = __shfl_sync(kFull, incl, 31);
        __syncwarp();
        uint32_t jc = 0;
        for (uint32_t c0 = 0; c0 < T; c0 += 32 * kLongUnroll - 1) {
          uint4 A[kLongUnroll];
          uint32_t jp[kLongUnroll];
#pragma unroll
          for (uint32_t u = 0; u < kLongUnroll; u++) {
            const uint32_t c = c0 + 32 * u + lane;
            jp[u] = 0xffffffffu;
            A[u] = make_uint4(0, 0, 0, 0);
            if (c < T) {
              while (gX[jc + 1] <= c) jc++;
              const uint32_t pc = c - gX[jc];
              jp[u] = jc | (pc << 5);
              const int64_t s0 = (int64_t)gS[jc] - (int64_t)(gD[jc] & 15);
              A[u] = ld16_abs<SEEK, kL1>(a, (s0 & ~(int64_t)15) + 16 * (int64_t)pc, b, obase);
            }
          }
#pragma unroll
          for (uint32_t u = 0; u < kLongUnroll; u++) {
            const uint4 nb = shfl_down16(A[u], 1);
            const uint32_t un = u + 1 < kLongUnroll ? u + 1 : u;
            const uint4 n0 = make_uint4(__shfl_sync(kFull, A[un].x, 0), __shfl_sync(kFull, A[un].y, 0),
                                        __shfl_sync(kFull, A[un].z, 0), __shfl_sync(kFull, A[un].w, 0));
            const uint4 B = lane == 31 ? n0 : nb;
            if (jp[u] == 0xffffffffu || (u + 1 == kLongUnroll && lane == 31)) continue;
            const uint32_t j = jp[u] & 31, pc = jp[u] >> 5, ml = gL[j];
            const uint32_t hd = gD[j] & 15;
            if (pc >= ((hd + ml + 15) >> 4)) continue;  // the trailing source piece stores nothing
            const uint4 v = funnel128(A[u], B, (uint32_t)(((int64_t)gS[j] - (int64_t)hd) & 15));
            uint8_t* dp = obase + gD[j] - hd + 16ull * pc;
            const int first = 16 * (int)pc - (int)hd;  // match byte held by the piece's first byte
            if (first >= 0 && first + 16 <= (int)ml)
              *reinterpret_cast<uint4*>(dp) = v;
            else
              store_bytes16(dp, v, (uint32_t)max(0, -first), (uint32_t)min(16, (int)ml - first));
          }
        }
        __syncwarp();
      }
      // the rest laid end to end in group order: gX[j] is where match j
      // starts, gX[kMatchGroup] the total
      const uint32_t bgo = go & ~sgo & ~lgo;
      if (!__any_sync(kFull, bgo != 0)) {  // none this round
        pend &= ~go;
        __syncwarp();  // the round's copies are seen by the next round's loads
        continue;
      }
      uint32_t carry = 0;
#pragma unroll
      for (uint32_t q = 0; q < kLaneMatches; q++) {
        const uint32_t j = lane + 32 * q;
        const uint32_t len = (bgo >> q & 1) ? gL[j] : 0u;
        const uint32_t incl = warp_incl_sum(len, lane);
        gX[j] = carry + incl - len;
        carry += __shfl_sync(kFull, incl, 31);
      }
      if (lane == 0) gX[kMatchGroup] = carry;
      __syncwarp();
      // lane l copies bytes c + 32 u + l: consecutive lanes read and write
      // consecutive bytes of a match, kCopyUnroll loads in flight before
      // their stores (a round's ready matches read no byte it writes); the
      // lane's match index only moves forward
      uint32_t jc = 0;
      for (uint32_t c = 0; c < carry; c += 32 * kCopyUnroll) {
        uint8_t v[kCopyUnroll];
        uint8_t* dp[kCopyUnroll];
#pragma unroll
        for (uint32_t u = 0; u < kCopyUnroll; u++) {
          const uint32_t p = c + 32 * u + lane;
          dp[u] = nullptr;
          if (p < carry) {
            while (gX[jc + 1] <= p) jc++;
            const uint32_t i = p - gX[jc], ml = gL[jc];
            const uint64_t S = gS[jc], d = bstart + gD[jc] - S;
            v[u] = ld_src<kL1>(Addr<SEEK>::at(a, src_index(S, d, ml, i), b, obase));
            dp[u] = obase + gD[jc] + i;
          }
        }
#pragma unroll
        for (uint32_t u = 0; u < kCopyUnroll; u++)
          if (dp[u]) *dp[u] = v[u];
      }
      pend &= ~go;
      __syncwarp();
    }
    if (!WAIT) {
#pragma unroll
      for (uint32_t q = 0; q < kLaneMatches; q++) {
        if (!(chk >> q & 1)) continue;
        if (f0[q] >= lvl || f1[q] >= lvl) bad = true;
        const uint32_t j = lane + 32 * q;
        const uint64_t S = gS[j], D = bstart + gD[j];
        const uint64_t rend = S + min((uint64_t)gL[j], D - S);
        const uint64_t k0 = S >> a.log2B, k1 = min((rend - 1) >> a.log2B, (uint64_t)b - 1);
        for (uint64_t k = k0 + 1; k < k1; k++)  // a source spanning more than two earlier blocks
          if (__ldg(a.level + k) >= lvl) bad = true;
      }
      if (__any_sync(kFull, bad)) fail(a, ok, ACE_E_CORRUPT, b, 39, lane);
      __syncwarp();
    }
  }
  cp_async_wait<0>();  // no record copy may land after the caller reuses the area
  __syncwarp();
  return ok;
}

// The three passes of a decode, each a persistent launch over the blocks:
// tokens (lengths, offsets, match records), literals, and matches.
// PASS_MATCH resolves blocks in (level, block) order with bounded waits on
// their source blocks (match_level_kernel resolves one level of a whole
// decode without them).
// PASS_FUSED runs all three for one block in one warp, block after block:
// tokens, then literals, then matches with bounded waits on the source
// blocks' flags, then the block's publication.  One launch covers the whole
// decode, so the issue-bound entropy decode of some warps overlaps the
// latency-bound match copies of others on the same SM.
enum { PASS_TOKENS = 0, PASS_LITERALS = 1, PASS_MATCH = 2, PASS_FUSED = 3 };

// Registers per thread allowed by each pass's launch bounds (256 threads).
#define ACE_PASS_MIN_CTAS(P) ((P) == PASS_TOKENS ? 4 : (P) == PASS_LITERALS ? 4 : (P) == PASS_FUSED ? 4 : 2)



// Publishes block b (its writes visible device-wide before the flag).
__device__ __forceinline__ void publish(uint32_t* ready, uint32_t b, uint32_t epoch, uint32_t lane) {
  __threadfence();
  __syncwarp();
  if (lane == 0) st_release(ready + b, epoch);
}

// Blocks level l of a fused call holds (whole decode: the index's level
// histogram; seek: the closure's level ranges in the scratch header).
template <bool SEEK>
__device__ __forceinline__ uint32_t level_size(const DecodeArgs& a, uint32_t l) {
  if (SEEK) return *(volatile uint32_t*)&a.sh->lv_start[l + 1] - *(volatile uint32_t*)&a.sh->lv_start[l];
  return __ldg(a.lv_count + l);
}

// The work of one archive (whole decode or seek): its list, in level order.
template <bool SEEK>
struct ArchiveJobs {
  const DecodeArgs& a;
  __device__ const DecodeArgs& job(uint32_t v, uint32_t& b) const {
    b = __ldg(a.items + v);
    return a;
  }
  __device__ uint32_t below(const DecodeArgs& x, uint32_t L) const { return level_size<SEEK>(x, L - 1); }
};

// Deferred match jobs a warp holds at most; warps per CTA at most.
constexpr uint32_t kDeferred = 4;
constexpr uint32_t kMaxWarps = 8;

// The fused schedule (Section 2's rule, a block decodes once the blocks its
// matches read are present, applied inside one launch).  Warps take blocks
// from the level-ordered list.  For each one a warp first decodes the
// entropy layer (length, offset and literal streams; literals placed at
// their output positions), then defers the block's match job until every
// block of the lower levels has its matches resolved (the level counters).
// A warp resolves its oldest deferred block as soon as that holds, and takes
// a new block while it waits, up to kDeferred held; so issue-bound entropy
// decode and latency-bound match copies of different warps share each SM
// and no warp idles while there is entropy work left.  With kDeferred held,
// or no blocks left, it waits (bounded, giving up on any recorded error).
// This always ends: the earliest unresolved block of the list has every
// lower level resolved (they come before it), and it is the oldest block of
// the warp holding it.
template <bool SEEK, class Jobs>
__device__ void fused_loop(const Jobs& jobs, ScratchHdr* sh, uint32_t n_items, uint64_t timeout_ns, uint8_t* wsm,
                           uint32_t lane, uint32_t epoch, uint32_t window) {
  uint32_t* const ticket = &sh->ticket;
  constexpr uint32_t ring = SEEK ? kSeekRing : kRing;
  // list positions of the warp's deferred blocks, a ring in shared memory
  // (registers are the scarce resource here): q[(q0 + k) % kDeferred]
  __shared__ uint32_t qs[kMaxWarps][kDeferred];
  uint32_t* const q = qs[threadIdx.x >> 5];
  uint32_t q0 = 0, nq = 0;
  bool more = true;  // blocks may remain in the list
  while (true) {
    if (*(volatile uint32_t*)&sh->status) break;
    if (nq) {
      uint32_t b;
      auto&& a = jobs.job(q[q0], b);
      const uint32_t L = __ldg(a.level + b);
      const uint32_t need = L ? jobs.below(a, L) : 0u;
      bool rdy = true;
      if (lane == 0 && L) rdy = ld_acquire(a.lv_done + L - 1) == need;
      rdy = __shfl_sync(kFull, rdy, 0);
      if (rdy || nq == kDeferred || !more) {
        if (!rdy) {  // nothing else to do: wait, bounded
          uint32_t ok = 1;
          if (lane == 0) {
            const uint64_t t0 = globaltimer();
            uint32_t ns = 32;
            while (ld_acquire(a.lv_done + L - 1) != need) {
              if (*(volatile uint32_t*)&sh->status) {
                ok = 0;
                break;
              }
              if (globaltimer() - t0 > timeout_ns) {
                record_error(&sh->status, &sh->err_block, &sh->err_where, ACE_E_TIMEOUT, b, 38);
                ok = 0;
                break;
              }
              __nanosleep(ns);
              if (ns < 1024) ns <<= 1;
            }
          }
          if (!__shfl_sync(kFull, ok, 0)) break;
        }
        // The bytes of the blocks below were written by other SMs.  Source
        // loads may still go through L1: a block's bytes are written by the
        // one warp that holds it, and read by other warps only after the
        // acquire below has seen its level complete, so no SM can hold an
        // older copy of them.
        fence_acquire();
        const uint32_t ntok = __ldg(reinterpret_cast<const uint32_t*>(a.dir + b) + 12);
        bool ok;
        if (SEEK) {
          // source blocks must be members of the closure; published ones
          // carry the epoch without the pending bit, so the flag checks do
          // not wait
          ok = match_block<true, true, true>(a, reinterpret_cast<MatchRec*>(wsm), b, lane, epoch,
                                             ntok ? ntok - 1 : 0);
          if (ok && a.slice) {
            uint64_t bs = (uint64_t)b << a.log2B, be = min(bs + ((uint64_t)1 << a.log2B), a.total);
            uint64_t lo = max(bs, a.coord), hi = min(be, a.coord + a.len);
            const uint8_t* src = a.out + slot_base(a, b) - bs;
            if (hi > lo) warp_copy(a.slice + (lo - a.coord), src + lo, hi - lo, lane);
          }
          if (ok) publish(a.ready, b, epoch, lane);
        } else {
          ok = match_block<false, false, true>(a, reinterpret_cast<MatchRec*>(wsm), b, lane, epoch,
                                               ntok ? ntok - 1 : 0, L);
        }
        if (!ok) break;  // the error is recorded; every warp stops
        __threadfence();
        __syncwarp();
        if (lane == 0) atomicAdd(a.lv_done + L, 1u);
        q0 = (q0 + 1) % kDeferred;
        nq--;
        continue;
      }
    }
    if (!more) {
      if (!nq) break;
      continue;
    }
    uint32_t u = 0;
    if (lane == 0) u = atomicAdd(ticket, 1u);
    u = __shfl_sync(kFull, u, 0);
    if (u >= n_items) {
      more = false;
      continue;
    }
    uint32_t b;
    auto&& a = jobs.job(u, b);
    bool ok = token_block<SEEK>(a, carve_tok(wsm), b, lane);
    if (ok) ok = literal_block<SEEK, ring>(a, carve_lit(wsm, window, ring), b, lane);
    if (!ok) break;
    if (lane == 0) q[(q0 + nq) % kDeferred] = u;
    __syncwarp();
    nq++;
  }
}

// One pass over a work list by persistent warps: the token pass decodes every
// block's length and offset streams into match records; the literal pass
// decodes every block's literal stream straight to its output positions; the
// match pass, launched after them, resolves every block's matches in (level,
// block) order, waiting on source blocks' flags, and publishes the block.
template <bool SEEK, int PASS>
__global__ void __launch_bounds__(256, ACE_PASS_MIN_CTAS(PASS)) decode_kernel(DecodeArgs a) {
  extern __shared__ __align__(16) uint8_t smem[];
  const uint32_t lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const uint32_t epoch = *(volatile uint32_t*)&a.sh->epoch;
  const uint32_t n_items = SEEK ? *(volatile uint32_t*)&a.sh->n_work : a.n_items;
  // the literal and match passes run only after every block's tokens decoded
  if (PASS != PASS_TOKENS && *(volatile uint32_t*)&a.sh->status) return;
  uint8_t* wsm = smem + (size_t)wid * a.warp_smem;
  if (PASS == PASS_FUSED) {
    fused_loop<SEEK>(ArchiveJobs<SEEK>{a}, a.sh, n_items, a.timeout_ns, wsm, lane, epoch, a.window);
    return;
  }
  uint32_t* ticket = PASS == PASS_TOKENS ? &a.sh->ticket : PASS == PASS_LITERALS ? &a.sh->ticket2 : &a.sh->ticket3;
  while (true) {
    uint32_t it = 0;
    if (lane == 0) it = atomicAdd(ticket, 1u);
    it = __shfl_sync(kFull, it, 0);
    if (it >= n_items) break;
    uint32_t b = __ldg(a.items + it);
    if (PASS == PASS_TOKENS) {
      token_block<SEEK>(a, carve_tok(wsm), b, lane);
      continue;
    }
    if (PASS == PASS_LITERALS) {
      constexpr uint32_t ring = SEEK ? kSeekRing : kRing;
      literal_block<SEEK, ring>(a, carve_lit(wsm, a.window, ring), b, lane);
      continue;
    }
    const uint32_t ntok = __ldg(reinterpret_cast<const uint32_t*>(a.dir + b) + 12);
    bool ok = match_block<SEEK, true>(a, reinterpret_cast<MatchRec*>(wsm), b, lane, epoch, ntok ? ntok - 1 : 0);
    if (SEEK && ok && a.slice) {
      // copy the part of this block inside [coord, coord + len) to the caller
      uint64_t bs = (uint64_t)b << a.log2B, be = min(bs + ((uint64_t)1 << a.log2B), a.total);
      uint64_t lo = max(bs, a.coord), hi = min(be, a.coord + a.len);
      const uint8_t* src = a.out + slot_base(a, b) - bs;
      if (hi > lo) warp_copy(a.slice + (lo - a.coord), src + lo, hi - lo, lane);
    }
    publish(a.ready, b, epoch, lane);
  }
}

// The match pass of one dependency level of a whole decode: every lower
// level was finished by the launches before, so blocks need no flags or
// waits.  Blocks are dealt out statically (block k of the level to warp
// k mod the warps in the grid), and each warp fetches its next block's
// number and record range while it resolves the current one.
__global__ void __launch_bounds__(256, 3) match_level_kernel(DecodeArgs a) {
  extern __shared__ __align__(16) uint8_t smem[];
  const uint32_t lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const uint32_t nw = gridDim.x * (blockDim.x >> 5);
  if (*(volatile uint32_t*)&a.sh->status) return;
  MatchRec* gm = reinterpret_cast<MatchRec*>(smem + (size_t)wid * kMatchSmem);
  uint32_t it = blockIdx.x * (blockDim.x >> 5) + wid;
  if (it >= a.n_items) return;
  auto n_matches = [&](uint32_t b) -> uint32_t {
    return (uint32_t)(__ldg(a.match_ptr + b + 1) - __ldg(a.match_ptr + b));
  };
  uint32_t b = __ldg(a.items + it);
  uint32_t nm = n_matches(b);
  while (true) {
    const uint32_t nx = it + nw;
    uint32_t bn = 0, nmn = 0;
    if (nx < a.n_items) {
      bn = __ldg(a.items + nx);
      nmn = n_matches(bn);
    }
    match_block<false, false>(a, gm, b, lane, 0, nm, a.cur_level);
    if (nx >= a.n_items) break;
    it = nx;
    b = bn;
    nm = nmn;
  }
}

// The match pass of a dependency level with few blocks, a CTA per block: a
// warp per block would leave most of the GPU idle while each block's matches
// resolve one round after another.  Every byte of the block gets a 16-bit
// entry in shared memory: 0x8000 | its value once final (a literal, or a
// match byte whose source lies in an earlier block, which the launches
// before finished), else the in-block position it copies.  A match byte
// equals the byte at its source, which precedes it (Section 2, the
// sequential LZ77 copy), so the entries form chains that each end at a final
// one; pointer jumping (every pending entry takes its target's entry) ends
// all of them in at most log2(B) + 1 sweeps.  The block is then written back
// with 16-byte stores.
constexpr uint32_t kSmallThreads = 512;
constexpr uint32_t kSmallMaxLog2B = 15;               // positions fit the entries' low 15 bits
constexpr uint32_t kSmallSweeps = kSmallMaxLog2B + 2;  // log2(B) + 1, and one that sees no pending entry
constexpr uint32_t kSmallUnroll = 8;                   // match bytes per lane with their loads in flight
constexpr uint32_t kSmallLoads = 4;                    // 16-byte block loads per thread in flight

// The CTA's current kSmallThreads matches (one record per thread), laid end
// to end: match j's bytes start at X[j], X[kSmallThreads] is their total.
struct __align__(16) SmallChunk {
  uint64_t S[kSmallThreads];
  uint32_t D[kSmallThreads], L[kSmallThreads], X[kSmallThreads + 1];
  uint32_t wsum[kSmallThreads / 32];
};

// One warp's current 32 matches, laid end to end (blocks of many matches).
struct __align__(16) SmallWarp {
  uint64_t S[32];
  uint32_t D[32], L[32], X[33];
};
// The entries, then the chunk's or the warps' arrays (one or the other per
// block): 43 KB for 16 KiB blocks, within the default shared-memory limit.
constexpr size_t kSmallArrays = sizeof(SmallChunk) > kSmallThreads / 32 * sizeof(SmallWarp)
                                    ? sizeof(SmallChunk)
                                    : kSmallThreads / 32 * sizeof(SmallWarp);
__host__ __device__ constexpr size_t small_smem_bytes(uint32_t log2B) {
  return ((size_t)2 << log2B) + kSmallArrays;
}

__global__ void __launch_bounds__(kSmallThreads, 1) match_small_kernel(DecodeArgs a) {
  extern __shared__ __align__(16) uint8_t smem[];
  const uint32_t tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  if (__syncthreads_or(*(volatile uint32_t*)&a.sh->status != 0)) return;  // the same answer for the whole CTA
  const uint32_t b = __ldg(a.items + blockIdx.x);
  const uint64_t B = 1ull << a.log2B, bstart = (uint64_t)b << a.log2B;
  const uint32_t blen = (uint32_t)min(B, a.total - bstart);
  uint8_t* obase = a.out + bstart;
  uint16_t* e = reinterpret_cast<uint16_t*>(smem);
  SmallChunk* const chunks = reinterpret_cast<SmallChunk*>(smem + (2ull << a.log2B));
  static_assert(sizeof(SmallChunk) % 16 == 0, "chunk arrays stay 16-byte aligned");
  const uint64_t m0 = __ldg(a.match_ptr + b), nm = __ldg(a.match_ptr + b + 1) - m0;
  const uint4* rec = reinterpret_cast<const uint4*>(a.recs + m0);
  bool bad = false;
  // the first chunk's match records load with the block
  uint4 rn = make_uint4(0, 0, 0, 0);
  if (tid < nm) rn = __ldg(rec + tid);

  // every byte final with what the literal pass left; match bytes are
  // overwritten next.  16-byte loads, kSmallLoads per thread in flight
  // (obase is block-aligned, and B is a multiple of 256).
  for (uint32_t j0 = 16 * tid; j0 < blen; j0 += 16 * kSmallThreads * kSmallLoads) {
    uint4 v[kSmallLoads];
#pragma unroll
    for (uint32_t u = 0; u < kSmallLoads; u++) {
      const uint32_t j = j0 + 16 * kSmallThreads * u;
      v[u] = make_uint4(0, 0, 0, 0);
      if (j + 16 <= blen) {
        v[u] = *reinterpret_cast<const uint4*>(obase + j);
      } else if (j < blen) {
        uint32_t x[4];
#pragma unroll
        for (uint32_t q = 0; q < 4; q++) {
          x[q] = 0;
#pragma unroll
          for (uint32_t k = 0; k < 4; k++)
            if (j + 4 * q + k < blen) x[q] |= (uint32_t)obase[j + 4 * q + k] << (8 * k);
        }
        v[u] = make_uint4(x[0], x[1], x[2], x[3]);
      }
    }
#pragma unroll
    for (uint32_t u = 0; u < kSmallLoads; u++) {
      const uint32_t j = j0 + 16 * kSmallThreads * u;
      if (j >= blen) continue;
      uint4* e4 = reinterpret_cast<uint4*>(e + j);
      e4[0] = make_uint4(__byte_perm(v[u].x, 0x80u, 0x4140), __byte_perm(v[u].x, 0x80u, 0x4342),
                         __byte_perm(v[u].y, 0x80u, 0x4140), __byte_perm(v[u].y, 0x80u, 0x4342));
      e4[1] = make_uint4(__byte_perm(v[u].z, 0x80u, 0x4140), __byte_perm(v[u].z, 0x80u, 0x4342),
                         __byte_perm(v[u].w, 0x80u, 0x4140), __byte_perm(v[u].w, 0x80u, 0x4342));
    }
  }
  __syncthreads();

  // match bytes: a byte whose source is in an earlier block reads it
  // (final), one whose source is in this block points there.  Blocks of at
  // most kSmallThreads matches lay them end to end over the whole CTA (every
  // thread on bytes tid, tid + kSmallThreads, ...); with more, each warp
  // takes 32 at a time on its own, without CTA barriers between them.
  if (nm > kSmallThreads) {
    SmallWarp& ww = reinterpret_cast<SmallWarp*>(chunks)[wid];
    for (uint64_t t0 = 32ull * wid; t0 < nm; t0 += kSmallThreads) {
      const uint64_t t = t0 + lane;
      const uint4 r = rn;
      if (t + kSmallThreads < nm) rn = __ldg(rec + t + kSmallThreads);  // the warp's next 32
      uint32_t len = 0;
      if (t < nm) {
        const uint64_t S = (uint64_t)r.x | ((uint64_t)r.y << 32);
        const uint32_t D = r.z, ml = r.w;
        if (ml && (S >= bstart + D || (uint64_t)D + ml > blen)) {
          bad = true;
        } else {
          len = ml;
        }
        ww.S[lane] = S;
        ww.D[lane] = D;
      }
      ww.L[lane] = len;
      const uint32_t incl = warp_incl_sum(len, lane);
      ww.X[lane] = incl - len;
      if (lane == 31) ww.X[32] = incl;
      const uint32_t total = __shfl_sync(kFull, incl, 31);
      __syncwarp();
      uint32_t jc = 0;  // the match of the lane's byte only moves forward
      for (uint32_t c = 0; c < total; c += 32 * kSmallUnroll) {
        uint32_t val[kSmallUnroll], dst[kSmallUnroll];
#pragma unroll
        for (uint32_t u = 0; u < kSmallUnroll; u++) {
          const uint32_t p = c + 32 * u + lane;
          dst[u] = ~0u;
          val[u] = 0;
          if (p < total) {
            while (ww.X[jc + 1] <= p) jc++;
            const uint32_t i = p - ww.X[jc], ml = ww.L[jc], D = ww.D[jc];
            const uint64_t S = ww.S[jc];
            const uint64_t src = src_index(S, bstart + D - S, ml, i);
            dst[u] = D + i;
            val[u] = src < bstart ? 0x8000u | ld_src<true>(a.out + src) : (uint32_t)(src - bstart);
          }
        }
#pragma unroll
        for (uint32_t u = 0; u < kSmallUnroll; u++)
          if (dst[u] != ~0u) e[dst[u]] = (uint16_t)val[u];
      }
      __syncwarp();  // the warp's next 32 reuse its arrays
    }
  }
  if (nm <= kSmallThreads && nm) {  // one chunk
    SmallChunk& w = chunks[0];
    const uint64_t t = tid;
    const uint4 r = rn;
    uint32_t len = 0;
    if (t < nm) {
      const uint64_t S = (uint64_t)r.x | ((uint64_t)r.y << 32);
      const uint32_t D = r.z, ml = r.w;
      if (ml && (S >= bstart + D || (uint64_t)D + ml > blen)) {
        bad = true;  // a source must precede its destination, which stays in the block
      } else {
        len = ml;
      }
      w.S[tid] = S;
      w.D[tid] = D;
    }
    w.L[tid] = len;
    // exclusive scan of the lengths over the CTA
    const uint32_t incl = warp_incl_sum(len, lane);
    if (lane == 31) w.wsum[wid] = incl;
    __syncthreads();
    uint32_t before = 0, total = 0;
#pragma unroll
    for (uint32_t k = 0; k < kSmallThreads / 32; k++) {
      const uint32_t x = w.wsum[k];
      before += k < wid ? x : 0u;
      total += x;
    }
    w.X[tid] = before + incl - len;
    if (tid == 0) w.X[kSmallThreads] = total;
    __syncthreads();
    for (uint32_t c = 0; c < total; c += kSmallThreads * kSmallUnroll) {
      uint32_t val[kSmallUnroll], dst[kSmallUnroll];
#pragma unroll
      for (uint32_t u = 0; u < kSmallUnroll; u++) {
        const uint32_t p = c + kSmallThreads * u + tid;
        dst[u] = ~0u;
        val[u] = 0;
        if (p < total) {
          const uint32_t jc = upper_bound(kSmallThreads + 1, p, [&](uint32_t i) { return w.X[i]; }) - 1;
          const uint32_t i = p - w.X[jc], ml = w.L[jc], D = w.D[jc];
          const uint64_t S = w.S[jc];
          const uint64_t src = src_index(S, bstart + D - S, ml, i);
          dst[u] = D + i;
          val[u] = src < bstart ? 0x8000u | ld_src<true>(a.out + src) : (uint32_t)(src - bstart);
        }
      }
#pragma unroll
      for (uint32_t u = 0; u < kSmallUnroll; u++)
        if (dst[u] != ~0u) e[dst[u]] = (uint16_t)val[u];
    }
  }
  if (__syncthreads_or(bad)) {
    if (tid == 0) record_error(&a.sh->status, &a.sh->err_block, &a.sh->err_where, ACE_E_CORRUPT, b, 39);
    return;
  }

  // pointer jumping; every target precedes its entry, so the sweeps end.
  // Entries change while others read them: each read sees an entry of the
  // same chain, old or new, and 16-bit shared stores do not tear.
  volatile uint16_t* ev = e;
  uint32_t sweep = 0;
  for (; sweep < kSmallSweeps; sweep++) {
    int pending = 0;
    for (uint32_t j = tid; j < blen; j += kSmallThreads) {
      const uint32_t x = ev[j];
      if (!(x & 0x8000u)) {
        const uint32_t y = ev[x];
        ev[j] = (uint16_t)y;
        pending |= !(y & 0x8000u);
      }
    }
    if (!__syncthreads_or(pending)) break;
  }
  if (sweep == kSmallSweeps) {  // cannot happen for the chains above
    if (tid == 0) record_error(&a.sh->status, &a.sh->err_block, &a.sh->err_where, ACE_E_CORRUPT, b, 42);
    return;
  }

  // the block's bytes: the low byte of each entry
  for (uint32_t j = 16 * tid; j < blen; j += 16 * kSmallThreads) {
    const uint4 lo = *reinterpret_cast<const uint4*>(e + j), hi = *reinterpret_cast<const uint4*>(e + j + 8);
    const uint4 v = make_uint4(__byte_perm(lo.x, lo.y, 0x6420), __byte_perm(lo.z, lo.w, 0x6420),
                               __byte_perm(hi.x, hi.y, 0x6420), __byte_perm(hi.z, hi.w, 0x6420));
    if (j + 16 <= blen) {
      *reinterpret_cast<uint4*>(obase + j) = v;
    } else {
      for (uint32_t k = 0; j + k < blen; k++) {
        const uint32_t x = k < 4 ? v.x : k < 8 ? v.y : k < 12 ? v.z : v.w;
        obase[j + k] = (uint8_t)(x >> (8 * (k & 3)));
      }
    }
  }

  // the earlier blocks a match reads (at most two) belong to lower levels:
  // checked last, since a corrupt archive fails the call whatever was written
  for (uint64_t t = tid; t < nm; t += kSmallThreads) {
    const uint4 r = __ldg(rec + t);
    const uint64_t S = (uint64_t)r.x | ((uint64_t)r.y << 32);
    const uint32_t D = r.z, ml = r.w;
    if (!ml || (S >> a.log2B) >= b) continue;
    const uint64_t rend = S + min((uint64_t)ml, bstart + D - S);
    const uint64_t k1 = min((rend - 1) >> a.log2B, (uint64_t)b - 1);
    for (uint64_t k = S >> a.log2B; k <= k1; k++)
      if (__ldg(a.level + k) >= a.cur_level) {
        record_error(&a.sh->status, &a.sh->err_block, &a.sh->err_where, ACE_E_CORRUPT, b, 39);
        return;
      }
  }
}

// ----------------------------------------------------------- batch decode

// One independent archive of a batch, as the batch kernel sees it.
struct ObjDesc {
  const uint8_t* arc;
  const ace_block_dir* dir;
  uint64_t payload_off;
  uint64_t total;
  uint8_t* out;
  uint32_t* ready;
  const uint32_t* order;  // the archive's blocks in (level, block) order
  const uint32_t* level;  // each block's dependency level
  MatchRec* recs;         // the archive's match records
  const uint64_t* match_ptr;
  uint32_t* lv_done;         // fused schedule: blocks of each level with matches resolved
  const uint32_t* lv_count;  // blocks per level
  uint32_t log2B, w, nb, pad;
};

struct BatchArgs {
  const ObjDesc* objs;
  const uint32_t* item_start;  // [n_objs + 1]: first work item of each archive
  uint32_t n_objs, n_items;
  uint32_t window, warp_smem, esc_cap, max_ntok;
  ScratchHdr* sh;
  uint64_t timeout_ns;
  uint32_t long_min;
};

// The work of a batch: (archive, block) items, each archive's blocks in its
// own level order.
struct BatchJobs {
  const BatchArgs& ba;
  __device__ uint32_t obj_of(uint32_t it) const {
    uint32_t lo = 0, hi = ba.n_objs;  // the archive o with item_start[o] <= it < item_start[o + 1]
    while (hi - lo > 1) {
      const uint32_t mid = (lo + hi) >> 1;
      if (__ldg(ba.item_start + mid) <= it) lo = mid;
      else hi = mid;
    }
    return lo;
  }
  __device__ DecodeArgs job(uint32_t v, uint32_t& b) const;
  __device__ uint32_t below(const DecodeArgs& x, uint32_t L) const { return __ldg(x.lv_count + L - 1); }
};

// Thousands of independent archives in one persistent launch per pass:
// warps take (archive, block) items from one ticket; each archive's items
// are in its own (level, block) order, so in the match pass a warp only
// ever waits on blocks of its archive that were handed out before its own.
__device__ DecodeArgs batch_args(const BatchArgs& ba, const ObjDesc& od) {
  DecodeArgs a{};
  a.arc = od.arc;
  a.dir = od.dir;
  a.payload_off = od.payload_off;
  a.total = od.total;
  a.nb = od.nb;
  a.log2B = od.log2B;
  a.w = od.w;
  a.window = ba.window;
  a.esc_cap = ba.esc_cap;
  a.warp_smem = ba.warp_smem;
  a.max_ntok = ba.max_ntok;
  a.out = od.out;
  a.sh = ba.sh;
  a.ready = od.ready;
  a.timeout_ns = ba.timeout_ns;
  a.recs = od.recs;
  a.match_ptr = od.match_ptr;
  a.level = od.level;
  a.lv_done = od.lv_done;
  a.lv_count = od.lv_count;
  a.long_min = ba.long_min;
  return a;
}

__device__ DecodeArgs BatchJobs::job(uint32_t v, uint32_t& b) const {
  const uint32_t o = obj_of(v);
  const ObjDesc od = ba.objs[o];
  b = __ldg(od.order + (v - __ldg(ba.item_start + o)));
  return batch_args(ba, od);
}

template <int PASS>
__global__ void __launch_bounds__(256, ACE_PASS_MIN_CTAS(PASS)) batch_decode_kernel(BatchArgs ba) {
  extern __shared__ __align__(16) uint8_t smem[];
  const uint32_t lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (PASS != PASS_TOKENS && PASS != PASS_FUSED && *(volatile uint32_t*)&ba.sh->status) return;
  uint8_t* wsm = smem + (size_t)wid * ba.warp_smem;
  const uint32_t epoch = *(volatile uint32_t*)&ba.sh->epoch;
  if (PASS == PASS_FUSED) {
    fused_loop<false>(BatchJobs{ba}, ba.sh, ba.n_items, ba.timeout_ns, wsm, lane, epoch, ba.window);
    return;
  }
  uint32_t* ticket = PASS == PASS_TOKENS ? &ba.sh->ticket : PASS == PASS_LITERALS ? &ba.sh->ticket2 : &ba.sh->ticket3;
  const BatchJobs jobs{ba};
  while (true) {
    uint32_t it = 0;
    if (lane == 0) it = atomicAdd(ticket, 1u);
    it = __shfl_sync(kFull, it, 0);
    if (it >= ba.n_items) break;
    uint32_t b;
    const DecodeArgs a = jobs.job(it, b);
    if (PASS == PASS_TOKENS) {
      token_block<false>(a, carve_tok(wsm), b, lane);
    } else if (PASS == PASS_LITERALS) {
      literal_block<false, kRing>(a, carve_lit(wsm, ba.window, kRing), b, lane);
    } else {
      const uint32_t ntok = __ldg(reinterpret_cast<const uint32_t*>(a.dir + b) + 12);
      match_block<false, true>(a, reinterpret_cast<MatchRec*>(wsm), b, lane, epoch, ntok ? ntok - 1 : 0);
      publish(a.ready, b, epoch, lane);
    }
  }
}

// ---------------------------------------------------------- seek closure

struct ClosureArgs {
  const uint32_t* dep_ptr;
  const uint32_t* dep_iv;
  ScratchHdr* sh;
  uint32_t* marks;   // one bit per block, all clear between calls
  uint32_t* front0;
  uint32_t* front1;
  uint32_t* work;
  uint32_t* slot_of;
  uint64_t nb;
  uint64_t first, last;  // target blocks
  uint64_t cap;          // slots available
  const uint32_t* level; // by levels: each block's dependency level (else null)
  uint32_t n_levels;
  uint32_t* ready;       // closure blocks get the call's epoch with kPendingFlag set
  uint32_t* lv_done;     // fused seeks: per-level counters, cleared here (null otherwise)
};

// The blocks a seek must decode: its target blocks and, transitively, every
// block their matches read (Section 2).  Breadth first from the targets, a
// warp per frontier block with its lanes over the block's dependency
// intervals; then an ordered compaction of the marked blocks gives each its
// slot, and the work list is ordered by dependency level (blocks of a level
// in ascending order) with the level ranges in the scratch header -- a valid
// decode order either way, since sources always precede.  One CTA.
__global__ void closure_kernel(ClosureArgs a) {
  __shared__ uint32_t n_next, s_min;
  __shared__ uint32_t wsum[32];
  __shared__ uint32_t carry;
  __shared__ uint32_t lcnt[kMaxLevelLaunches + 1];
  const uint32_t tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
  if (tid == 0) {
    const uint32_t e = (a.sh->epoch + 1) & ~kPendingFlag;  // never 0, never with the pending bit
    a.sh->epoch = e ? e : 1u;
    a.sh->ticket = 0;
    a.sh->ticket2 = 0;
    a.sh->ticket3 = 0;
    s_min = (uint32_t)a.first;
  }
  if (tid <= kMaxLevelLaunches) {
    lcnt[tid] = 0;
    if (a.lv_done) a.lv_done[tid] = 0;
  }
  uint32_t ntar = (uint32_t)(a.last - a.first + 1);
  for (uint32_t i = tid; i < ntar; i += blockDim.x) {
    uint32_t b = (uint32_t)a.first + i;
    atomicOr(&a.marks[b >> 5], 1u << (b & 31));
    a.front0[i] = b;
  }
  uint32_t n_front = ntar;
  uint32_t* cur = a.front0;
  uint32_t* nxt = a.front1;
  __syncthreads();
  while (n_front) {
    if (tid == 0) n_next = 0;
    __syncthreads();
    for (uint32_t f = wid; f < n_front; f += nw) {
      const uint32_t b = cur[f];
      const uint32_t e1 = a.dep_ptr[b + 1];
      for (uint32_t e = a.dep_ptr[b] + lane; e < e1; e += 32) {
        const uint32_t k0 = a.dep_iv[2 * e], k1 = a.dep_iv[2 * e + 1];
        for (uint32_t k = k0; k <= k1; k++) {
          uint32_t old = atomicOr(&a.marks[k >> 5], 1u << (k & 31));
          if (!(old & (1u << (k & 31)))) {
            nxt[atomicAdd(&n_next, 1u)] = k;
            atomicMin(&s_min, k);
          }
        }
      }
    }
    __syncthreads();
    n_front = n_next;
    uint32_t* t = cur;
    cur = nxt;
    nxt = t;
    __syncthreads();
  }
  // ordered compaction of the marked blocks into front0, clearing the marks
  // behind it; a block's slot is its place in ascending order
  if (tid == 0) carry = 0;
  __syncthreads();
  uint32_t w0 = s_min >> 5, w1 = (uint32_t)(a.last >> 5);
  for (uint32_t c0 = w0; c0 <= w1; c0 += blockDim.x) {
    uint32_t wi = c0 + tid;
    uint32_t bits = wi <= w1 ? a.marks[wi] : 0u;
    uint32_t cnt = __popc(bits);
    uint32_t incl = warp_incl_sum(cnt, lane);
    if (lane == 31) wsum[wid] = incl;
    __syncthreads();
    if (wid == 0) {
      uint32_t s = lane < nw ? wsum[lane] : 0;
      uint32_t si = warp_incl_sum(s, lane);
      if (lane < nw) wsum[lane] = si - s;
    }
    __syncthreads();
    uint32_t pos = carry + wsum[wid] + incl - cnt;
    while (bits) {
      uint32_t bit = __ffs(bits) - 1;
      bits &= bits - 1;
      uint32_t b = wi * 32 + bit;
      if (pos < a.cap) {
        a.front0[pos] = b;
        a.slot_of[b] = pos;
      }
      pos++;
    }
    if (wi <= w1) a.marks[wi] = 0;
    __syncthreads();
    if (tid == blockDim.x - 1) carry = pos;
    __syncthreads();
  }
  const uint32_t n = carry;
  if (n > a.cap) {
    if (tid == 0) {
      record_error(&a.sh->status, &a.sh->err_block, &a.sh->err_where, ACE_E_NOMEM, n, 50);
      a.sh->n_work = 0;
    }
    return;
  }
  // the work list by level (one level when levels are not used)
  const uint32_t epoch = a.sh->epoch;
  for (uint32_t i = tid; i < n; i += blockDim.x) {
    const uint32_t b = a.front0[i];
    atomicAdd(&lcnt[a.level ? a.level[b] : 0], 1u);
    if (a.ready) a.ready[b] = epoch | kPendingFlag;  // a member of this seek's closure, not yet decoded
  }
  __syncthreads();
  if (tid == 0) {
    const uint32_t nl = a.level ? a.n_levels : 1;
    uint32_t c = 0;
    for (uint32_t l = 0; l < nl; l++) {
      const uint32_t k = lcnt[l];
      lcnt[l] = c;
      a.sh->lv_start[l] = c;
      c += k;
    }
    a.sh->lv_start[nl] = c;
    a.sh->n_work = n;
  }
  __syncthreads();
  for (uint32_t i = tid; i < n; i += blockDim.x) {
    const uint32_t b = a.front0[i];
    a.work[atomicAdd(&lcnt[a.level ? a.level[b] : 0], 1u)] = b;
  }
}

// ------------------------------------------------------ seek batches (cache)

// One archive attached to a decoded-block cache.
struct CacheArc {
  const uint8_t* arc;
  const ace_block_dir* dir;
  uint64_t payload_off;
  uint64_t total;
  const uint32_t* dep_ptr;
  const uint32_t* dep_iv;
  uint32_t* ready;    // == cache epoch: the block sits decoded in its slot
  uint32_t* slot_of;
  uint32_t* marks;    // closure marks, clear between calls
  uint32_t* wpos;     // a block decoded by the current batch: its place in the work list
  uint32_t nb, w;
};

// Header of a cache (first 256 bytes of its memory).
struct CacheHdr {
  uint32_t status, err_block, err_where;
  uint32_t epoch;      // blocks whose ready flag equals it are cached
  uint32_t ticket;
  uint32_t n_work;
  uint32_t n_cached;   // slots holding a decoded block
  uint32_t n_front;
  uint32_t hand;       // clock hand: the next slot the allocation looks at
  uint32_t serial;     // batches run: the slots a batch uses carry its serial
  uint64_t evicted;    // cached blocks evicted to make room, since creation
  uint32_t ticket2;    // next work item of the literal pass
  uint32_t ticket3;    // next work item of the match pass
  uint64_t decoded;    // blocks decoded, since creation
  uint32_t pad[48];
};
static_assert(sizeof(CacheHdr) == 256, "cache header");
static_assert(offsetof(CacheHdr, ticket2) == offsetof(ScratchHdr, ticket2), "shared header fields");
static_assert(offsetof(CacheHdr, ticket3) == offsetof(ScratchHdr, ticket3), "shared header fields");
static_assert(offsetof(CacheHdr, epoch) == offsetof(ScratchHdr, epoch), "shared header fields");
static_assert(offsetof(CacheHdr, ticket) == offsetof(ScratchHdr, ticket), "shared header fields");
static_assert(offsetof(CacheHdr, n_work) == offsetof(ScratchHdr, n_work), "shared header fields");

struct CacheArgs {
  CacheHdr* h;
  const CacheArc* arcs;
  uint32_t n_arcs;
  uint32_t log2B;
  uint32_t n_slots;
  uint32_t front_cap;    // blocks one batch may decode (work items), and the frontier's capacity
  uint32_t* front0;      // (archive, block) pairs
  uint32_t* front1;
  uint32_t* work;        // (archive, block) pairs in decode order
  uint32_t* taken;       // the slots the allocation took, one per work item
  uint32_t* arc_minmax;  // per archive: smallest, largest block marked
  uint32_t* owner_arc;   // per slot: the archive and block it holds (archive ~0: none)
  uint32_t* owner_blk;
  uint32_t* ref;         // per slot: the clock's reference bit
  uint32_t* use;         // per slot: the serial of the last batch that used it
  uint8_t* slots;
  MatchRec* recs;        // max_ntok match records per work item
  const ace_seek_req* reqs;
  uint32_t n_reqs;
};

// A block the batch needs: a cached one has its slot kept from eviction for
// this batch and its reference bit set (true: nothing to decode); an
// uncached one is marked for decoding (returns whether it was newly marked).
__device__ __forceinline__ bool cache_visit(const CacheArgs& c, uint32_t a, uint32_t b, uint32_t epoch,
                                            uint32_t serial, bool& cached) {
  const CacheArc& ca = c.arcs[a];
  // flags are set by earlier launches on this stream, ordered before this one
  cached = ld_relaxed(ca.ready + b) == epoch;
  if (cached) {
    const uint32_t sl = ca.slot_of[b];
    if (sl < c.n_slots) {
      c.use[sl] = serial;
      c.ref[sl] = 1;
    }
    return false;
  }
  const uint32_t bit = 1u << (b & 31);
  return !(atomicOr(ca.marks + (b >> 5), bit) & bit);
}

// The blocks a batch of seeks must decode: every target block that is not
// cached and, transitively, every uncached block their matches read
// (Section 2), listed archive by archive in ascending block order.  Each
// gets a slot from a clock over the slots: slots this batch uses are passed
// over, a slot whose reference bit is set gets a second chance (the bit is
// cleared), and a slot taken from a cached block evicts it.  One CTA.
__global__ void cache_closure_kernel(CacheArgs c) {
  __shared__ uint32_t n_next, carry, overflow, s_serial;
  __shared__ uint32_t s_taken, s_hand, s_scanned, s_stop;
  __shared__ uint32_t wsum[32];
  const uint32_t tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
  const uint32_t epoch = c.h->epoch;
  if (tid == 0) {
    n_next = 0;
    overflow = 0;
    s_serial = c.h->serial + 1;
    c.h->serial = s_serial;
  }
  for (uint32_t a = tid; a < c.n_arcs; a += blockDim.x) {
    c.arc_minmax[2 * a] = 0xffffffffu;
    c.arc_minmax[2 * a + 1] = 0;
  }
  __syncthreads();
  const uint32_t serial = s_serial;
  // targets: a thread per request
  for (uint32_t r = tid; r < c.n_reqs; r += blockDim.x) {
    const ace_seek_req q = c.reqs[r];
    uint64_t first = q.coord >> c.log2B, last = (q.coord + q.len - 1) >> c.log2B;
    for (uint64_t b = first; b <= last; b++) {
      bool cached;
      if (cache_visit(c, q.archive, (uint32_t)b, epoch, serial, cached)) {
        uint32_t i = atomicAdd(&n_next, 1u);
        if (i < c.front_cap) {
          c.front0[2 * i] = q.archive;
          c.front0[2 * i + 1] = (uint32_t)b;
        } else {
          overflow = 1;
        }
        atomicMin(&c.arc_minmax[2 * q.archive], (uint32_t)b);
        atomicMax(&c.arc_minmax[2 * q.archive + 1], (uint32_t)b);
      }
    }
  }
  __syncthreads();
  uint32_t n_front = min(n_next, c.front_cap);
  uint32_t* cur = c.front0;
  uint32_t* nxt = c.front1;
  __syncthreads();
  while (n_front && !overflow) {
    if (tid == 0) n_next = 0;
    __syncthreads();
    for (uint32_t i = wid; i < n_front; i += nw) {  // a warp per frontier block, lanes over its intervals
      uint32_t a = cur[2 * i], b = cur[2 * i + 1];
      const CacheArc& ca = c.arcs[a];
      const uint32_t e1 = ca.dep_ptr[b + 1];
      for (uint32_t e = ca.dep_ptr[b] + lane; e < e1; e += 32)
        for (uint32_t k = ca.dep_iv[2 * e]; k <= ca.dep_iv[2 * e + 1]; k++) {
          bool cached;
          if (cache_visit(c, a, k, epoch, serial, cached)) {
            uint32_t j = atomicAdd(&n_next, 1u);
            if (j < c.front_cap) {
              nxt[2 * j] = a;
              nxt[2 * j + 1] = k;
            } else {
              overflow = 1;
            }
            atomicMin(&c.arc_minmax[2 * a], k);
          }
        }
    }
    __syncthreads();
    n_front = min(n_next, c.front_cap);
    uint32_t* t = cur;
    cur = nxt;
    nxt = t;
    __syncthreads();
  }
  // ordered compaction into the work list, archive by archive, clearing the
  // marks behind it
  if (tid == 0) carry = 0;
  __syncthreads();
  for (uint32_t a = 0; a < c.n_arcs; a++) {
    uint32_t lo = c.arc_minmax[2 * a], hi = c.arc_minmax[2 * a + 1];
    if (lo > hi) continue;
    const CacheArc& ca = c.arcs[a];
    for (uint32_t c0 = lo >> 5; c0 <= (hi >> 5); c0 += blockDim.x) {
      uint32_t wi = c0 + tid;
      uint32_t bits = wi <= (hi >> 5) ? ca.marks[wi] : 0u;
      uint32_t cnt = __popc(bits);
      uint32_t incl = warp_incl_sum(cnt, lane);
      if (lane == 31) wsum[wid] = incl;
      __syncthreads();
      if (wid == 0) {
        uint32_t v = lane < nw ? wsum[lane] : 0;
        uint32_t vi = warp_incl_sum(v, lane);
        if (lane < nw) wsum[lane] = vi - v;
      }
      __syncthreads();
      uint32_t pos = carry + wsum[wid] + incl - cnt;
      while (bits) {
        uint32_t bit = __ffs(bits) - 1;
        bits &= bits - 1;
        uint32_t b = wi * 32 + bit;
        if (pos < c.front_cap) {
          c.work[2 * pos] = a;
          c.work[2 * pos + 1] = b;
        }
        pos++;
      }
      if (wi <= (hi >> 5)) ca.marks[wi] = 0;
      __syncthreads();
      if (tid == blockDim.x - 1) carry = pos;
      __syncthreads();
    }
  }
  const uint32_t n = carry;
  if (tid == 0) {
    s_taken = 0;
    s_hand = c.h->hand;
    s_scanned = 0;
  }
  __syncthreads();
  // the clock: at most two turns over the slots (after one, every bit of a
  // slot this batch does not use is clear)
  const uint64_t limit = overflow || n > c.front_cap ? 0ull : 2ull * c.n_slots;
  while (true) {
    const uint32_t taken = s_taken, hand = s_hand, scanned = s_scanned;
    if (taken >= n || scanned >= limit) break;
    const uint64_t room = limit - scanned;
    const uint32_t win = (uint32_t)min(min((uint64_t)blockDim.x, (uint64_t)c.n_slots), room);
    const uint32_t sl = (uint32_t)(((uint64_t)hand + tid) % c.n_slots);
    bool pinned = false, refd = false, elig = false;
    if (tid < win) {
      pinned = c.use[sl] == serial;
      refd = c.ref[sl] != 0;
      elig = !pinned && !refd;
    }
    const uint32_t e = elig ? 1u : 0u;
    const uint32_t incl = warp_incl_sum(e, lane);
    if (lane == 31) wsum[wid] = incl;
    __syncthreads();
    if (wid == 0) {
      uint32_t v = lane < nw ? wsum[lane] : 0;
      uint32_t vi = warp_incl_sum(v, lane);
      if (lane < nw) wsum[lane] = vi - v;
      if (lane == nw - 1) s_stop = vi;  // the window's eligible total, for a moment
    }
    __syncthreads();
    const uint32_t total = s_stop, rank = wsum[wid] + incl - e, rem = n - taken;
    __syncthreads();
    // the hand stops just after the rem-th eligible slot, else at the window's end
    if (total >= rem) {
      if (elig && rank == rem - 1) s_stop = tid;
    } else if (tid == 0) {
      s_stop = win - 1;
    }
    __syncthreads();
    const uint32_t stop = s_stop;
    if (tid <= stop && tid < win) {
      if (!pinned && refd) c.ref[sl] = 0;  // second chance
      if (elig && rank < rem) {
        c.taken[taken + rank] = sl;
        c.use[sl] = serial;  // taken: the next turn of the hand passes it over
      }
    }
    __syncthreads();
    if (tid == 0) {
      s_taken = taken + min(total, rem);
      s_hand = (uint32_t)(((uint64_t)hand + stop + 1) % c.n_slots);
      s_scanned = scanned + stop + 1;
    }
    __syncthreads();
  }
  const bool fits = !overflow && n <= c.front_cap && s_taken >= n;
  // each work item into its slot, evicting the slot's cached block
  if (fits) {
    for (uint32_t i = tid; i < n; i += blockDim.x) {
      const uint32_t sl = c.taken[i], a = c.work[2 * i], b = c.work[2 * i + 1];
      const uint32_t oa = c.owner_arc[sl], ob = c.owner_blk[sl];
      if (oa < c.n_arcs) {
        const CacheArc& o = c.arcs[oa];
        if (o.slot_of[ob] == sl && o.ready[ob] == epoch) {
          o.ready[ob] = 0;
          atomicAdd(reinterpret_cast<unsigned long long*>(&c.h->evicted), 1ull);
        }
      } else {
        atomicAdd(&c.h->n_cached, 1u);
      }
      c.owner_arc[sl] = a;
      c.owner_blk[sl] = b;
      c.use[sl] = serial;
      c.ref[sl] = 1;
      const CacheArc& ca = c.arcs[a];
      ca.slot_of[b] = sl;
      ca.wpos[b] = i;
    }
  }
  __syncthreads();
  if (tid == 0) {
    c.h->hand = s_hand;
    uint32_t nn = n;
    if (!fits) {
      record_error(&c.h->status, &c.h->err_block, &c.h->err_where, ACE_E_NOMEM, n, 51);
      nn = 0;
    } else {
      c.h->decoded += n;
    }
    c.h->n_work = nn;
    c.h->ticket = 0;
    c.h->ticket2 = 0;
    c.h->ticket3 = 0;
  }
}

struct CacheDecodeArgs {
  CacheArgs c;
  uint32_t window, warp_smem, esc_cap, max_ntok;
  uint64_t timeout_ns;
  uint32_t long_min;
};

// Decodes a batch's work list into cache slots: the same three passes as a
// seek, archive by archive.
template <int PASS>
__global__ void __launch_bounds__(256, ACE_PASS_MIN_CTAS(PASS)) cache_decode_kernel(CacheDecodeArgs ca) {
  extern __shared__ __align__(16) uint8_t smem[];
  const uint32_t lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  uint8_t* wsm = smem + (size_t)wid * ca.warp_smem;
  const CacheArgs& c = ca.c;
  if (PASS != PASS_TOKENS && *(volatile uint32_t*)&c.h->status) return;
  const uint32_t epoch = *(volatile uint32_t*)&c.h->epoch;
  const uint32_t n_items = *(volatile uint32_t*)&c.h->n_work;
  uint32_t* ticket = PASS == PASS_TOKENS ? &c.h->ticket : PASS == PASS_LITERALS ? &c.h->ticket2 : &c.h->ticket3;
  while (true) {
    uint32_t it = 0;
    if (lane == 0) it = atomicAdd(ticket, 1u);
    it = __shfl_sync(kFull, it, 0);
    if (it >= n_items) break;
    const uint32_t ai = __ldg(c.work + 2 * it), b = __ldg(c.work + 2 * it + 1);
    const CacheArc& arc = c.arcs[ai];
    DecodeArgs a{};
    a.arc = arc.arc;
    a.dir = arc.dir;
    a.payload_off = arc.payload_off;
    a.total = arc.total;
    a.nb = arc.nb;
    a.log2B = c.log2B;
    a.w = arc.w;
    a.window = ca.window;
    a.esc_cap = ca.esc_cap;
    a.warp_smem = ca.warp_smem;
    a.max_ntok = ca.max_ntok;
    a.out = c.slots;
    a.sh = reinterpret_cast<ScratchHdr*>(c.h);
    a.ready = arc.ready;
    a.slot_of = arc.slot_of;
    a.n_slots = c.n_slots;
    a.rec_index = arc.wpos;
    a.n_rec_slots = c.front_cap;
    a.long_min = ca.long_min;
    a.timeout_ns = ca.timeout_ns;
    a.recs = c.recs;
    a.match_ptr = nullptr;
    if (PASS == PASS_TOKENS) {
      token_block<true>(a, carve_tok(wsm), b, lane);
    } else if (PASS == PASS_LITERALS) {
      literal_block<true, kSeekRing>(a, carve_lit(wsm, ca.window, kSeekRing), b, lane);
    } else {
      const uint32_t ntok = __ldg(reinterpret_cast<const uint32_t*>(a.dir + b) + 12);
      match_block<true, true>(a, reinterpret_cast<MatchRec*>(wsm), b, lane, epoch, ntok ? ntok - 1 : 0);
      publish(arc.ready, b, epoch, lane);
    }
  }
}

// Each request's bytes from the cache slots to its place in the output pool.
__global__ void cache_copy_kernel(CacheArgs c, uint8_t* pool) {
  if (*(volatile uint32_t*)&c.h->status) return;  // a failed batch copies nothing
  const uint32_t lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const uint64_t B = (uint64_t)1 << c.log2B;
  for (uint32_t r = blockIdx.x; r < c.n_reqs; r += gridDim.x) {
    const ace_seek_req q = c.reqs[r];
    const CacheArc& ca = c.arcs[q.archive];
    if (q.len == 0) continue;
    // a warp per block the request covers: one slot lookup, then a batched copy
    const uint64_t k0 = q.coord >> c.log2B, k1 = (q.coord + q.len - 1) >> c.log2B;
    for (uint64_t k = k0 + wid; k <= k1; k += nw) {
      const uint64_t lo = max(k << c.log2B, q.coord), hi = min((k + 1) << c.log2B, q.coord + q.len);
      const uint32_t slot = __ldg(ca.slot_of + k);
      warp_copy(pool + q.out_off + (lo - q.coord), c.slots + ((uint64_t)slot << c.log2B) + (lo & (B - 1)), hi - lo,
                lane);
    }
  }
}

// New cache epoch: every cached block is forgotten, every slot is free
// (owners left behind no longer match their blocks' flags).
__global__ void cache_reset_kernel(CacheHdr* h) {
  h->epoch += 1;
  h->n_cached = 0;
  h->hand = 0;
  h->ticket = 0;
  h->ticket2 = 0;
  h->ticket3 = 0;
  h->n_work = 0;
}

// ------------------------------------------------------------ verification

__device__ __forceinline__ uint8_t pattern_byte(uint32_t seed, uint64_t i) {
  uint64_t z = (i + 1) * 0x9e3779b97f4a7c15ull ^ ((uint64_t)seed << 32 | seed);
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return (uint8_t)(z ^ (z >> 31));
}

__global__ void fill_pattern_kernel(uint8_t* p, uint64_t n, uint32_t seed) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
    p[i] = pattern_byte(seed, i);
}

__global__ void count_pattern_mismatch_kernel(const uint8_t* p, uint64_t n, uint32_t seed, uint64_t* bad) {
  uint64_t c = 0;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
    c += p[i] != pattern_byte(seed, i);
  if (c) atomicAdd((unsigned long long*)bad, (unsigned long long)c);
}

// New call on a scratch buffer: next epoch, ticket back to zero.
__global__ void begin_call_kernel(ScratchHdr* sh) {
  const uint32_t e = (sh->epoch + 1) & ~kPendingFlag;  // never 0, never with the pending bit
  sh->epoch = e ? e : 1u;
  sh->ticket = 0;
  sh->ticket2 = 0;
  sh->ticket3 = 0;
}

// FNV-1a 64 (Fowler/Noll/Vo): sequential by definition, one thread.  The
// bytes arrive in aligned 16-byte vectors, kFnvBatch at a time, the next
// batch's loads issued before the current batch is hashed, so the hash chain
// rather than the load latency sets the time.  The state is kept as two
// 32-bit halves: with the prime P = 2^40 + 0x1b3, h P mod 2^64 has low word
// (lo 0x1b3) mod 2^32 and high word ((lo 0x1b3) >> 32) + hi 0x1b3 + (lo << 8),
// so the chain from byte to byte runs through the low word alone.
constexpr uint32_t kFnvBatch = 8;
__global__ void fnv_kernel(const uint8_t* p, uint64_t n, uint64_t* out) {
  uint32_t lo = 0x84222325u, hi = 0xcbf29ce4u;  // the 64-bit offset basis
  auto step = [&](uint32_t b) {
    lo ^= b;
    hi = hi * 0x1b3u + __umulhi(lo, 0x1b3u) + (lo << 8);  // beside the low word's chain
    lo *= 0x1b3u;
  };
  uint64_t i = 0;
  for (; i < n && (reinterpret_cast<uintptr_t>(p + i) & 15); i++) step(p[i]);
  const uint4* v = reinterpret_cast<const uint4*>(p + i);
  const uint64_t nb = (n - i) / (16 * kFnvBatch);  // whole batches
  uint4 cur[kFnvBatch], nxt[kFnvBatch];
#pragma unroll
  for (uint32_t k = 0; k < kFnvBatch; k++) cur[k] = nb ? v[k] : make_uint4(0, 0, 0, 0);
  for (uint64_t q = 0; q < nb; q++) {
#pragma unroll
    for (uint32_t k = 0; k < kFnvBatch; k++) nxt[k] = q + 1 < nb ? v[(q + 1) * kFnvBatch + k] : cur[k];
#pragma unroll
    for (uint32_t k = 0; k < kFnvBatch; k++) {
      const uint32_t w[4] = {cur[k].x, cur[k].y, cur[k].z, cur[k].w};
#pragma unroll
      for (uint32_t j = 0; j < 16; j++) step((w[j >> 2] >> (8 * (j & 3))) & 0xffu);
    }
#pragma unroll
    for (uint32_t k = 0; k < kFnvBatch; k++) cur[k] = nxt[k];
  }
  for (i += nb * 16 * kFnvBatch; i < n; i++) step(p[i]);
  *out = ((uint64_t)hi << 32) | lo;
}

}  // namespace

// ---------------------------------------------------------------- host side

struct ace_index {
  const uint8_t* d_arc;
  uint64_t arc_bytes;
  ace_file_header h;
  uint8_t* d_mem;
  uint64_t mem_bytes;
  IndexHdr* d_ih;
  uint32_t* d_level;
  uint32_t* d_order;
  const uint32_t* d_dep_ptr;
  const uint32_t* d_dep_iv;
  uint64_t n_iv;
  uint32_t n_levels;
  uint32_t max_ntok;
  uint64_t n_matches;
  uint64_t* d_match_ptr;
  uint32_t* d_lv_count;  // blocks per level
  int device;
  int num_sms;
  ace_tune tune;
  // occupancy of the decode kernels, per (seek?, pass, warps per CTA, window)
  mutable int occ_cache[2][4][9][9];  // [3]: the fused pass
  mutable int occ_level[9][9];  // the per-level match kernel
  mutable bool small_attr = false;  // match_small_kernel allowed its shared memory
  // whole decodes resolve matches with one launch per level when there are
  // at most kMaxLevelLaunches levels: level L's blocks are
  // order[level_start[L] .. level_start[L + 1])
  bool by_levels;
  uint32_t level_start[kMaxLevelLaunches + 1];
};

namespace {

struct IndexLayout {
  uint64_t level, order, lv_count, lv_cursor, match_ptr, seen, total;
};

IndexLayout index_layout(uint64_t nb) {
  IndexLayout L;
  uint64_t o = sizeof(IndexHdr);
  L.level = o;
  o = align256(o + 4 * nb);
  L.order = o;
  o = align256(o + 4 * nb);
  L.lv_count = o;
  o = align256(o + 4 * (nb + 1));
  L.lv_cursor = o;
  o = align256(o + 4 * (nb + 1));
  L.match_ptr = o;
  o = align256(o + 8 * (nb + 1));
  L.seen = o;  // a stored index's order check marks each block here
  o = align256(o + 4 * nb);
  L.total = o;
  return L;
}

struct ScratchLayout {
  uint64_t ready, slot_of, work, marks, front0, front1, lv_done, tail, total;
};

// Bytes one seek slot needs: the decoded block and its match records.
inline uint64_t slot_bytes(uint32_t log2B, uint64_t max_ntok) {
  return (1ull << log2B) + 16 * max_ntok;
}

constexpr uint32_t kMaxWindow = 256;
constexpr uint32_t kMaxWarpsPerCta = 8;  // the decode kernel's launch bounds: 256 threads

// One layout serves every call on a scratch buffer, so whole decodes and
// seeks may share it: header, ready flags, the seek's slot map, work list,
// closure marks and frontiers, the fused schedule's level counters, then a
// tail that a whole decode uses for the archive's match records and a seek
// for its block slots followed by their match records.
ScratchLayout scratch_layout(uint64_t nb, uint32_t log2B, uint64_t max_seek, uint64_t max_ntok,
                             uint64_t n_matches) {
  ScratchLayout L;
  uint64_t o = sizeof(ScratchHdr);
  L.ready = o;
  o = align256(o + 4 * nb);
  L.slot_of = o;
  o = align256(o + 4 * nb);
  L.work = o;
  o = align256(o + 4 * nb);
  L.marks = o;
  o = align256(o + 4 * ((nb + 31) / 32));
  L.front0 = o;
  o = align256(o + 4 * nb);
  L.front1 = o;
  o = align256(o + 4 * nb);
  L.lv_done = o;
  o = align256(o + 4 * (nb + 1));
  L.tail = o;
  o = align256(o + std::max<uint64_t>(16 * n_matches, max_seek * slot_bytes(log2B, max_ntok)));
  L.total = o;
  return L;
}

ace_status parse_header(const void* h_header, uint64_t header_bytes, ace_file_header* h) {
  if (!h_header || header_bytes < sizeof(ace_file_header)) return ACE_E_INVAL;
  std::memcpy(h, h_header, sizeof *h);
  if (h->magic != ACE_MAGIC || h->version != ACE_VERSION || h->n_streams != ACE_NSTREAMS ||
      h->n_states != ACE_NSTATES || h->scale_bits != ACE_SCALE_BITS)
    return ACE_E_CORRUPT;
  if (h->off_width != 4 && h->off_width != 5) return ACE_E_CORRUPT;
  if (h->log2_block < ACE_MIN_LOG2_BLOCK || h->log2_block > ACE_MAX_LOG2_BLOCK) return ACE_E_CORRUPT;
  uint64_t B = 1ull << h->log2_block;
  if (h->n_blocks != (h->total_size + B - 1) / B || h->n_blocks > 0xFFFFFFF0ull) return ACE_E_CORRUPT;
  if (h->dir_off < sizeof(ace_file_header) || h->dir_off + h->n_blocks * sizeof(ace_block_dir) > h->deps_off)
    return ACE_E_CORRUPT;
  if (h->deps_off + 4 * (h->n_blocks + 1) > h->payload_off || h->payload_off > h->archive_bytes)
    return ACE_E_CORRUPT;
  if ((h->dir_off & 7) || (h->deps_off & 3) || (h->payload_off & 15) || (h->archive_bytes & 15))
    return ACE_E_CORRUPT;
  return ACE_OK;
}

inline bool aligned(const void* p, uintptr_t a) { return (reinterpret_cast<uintptr_t>(p) & (a - 1)) == 0; }

#define CUDA_TRY(x)                         \
  do {                                      \
    if ((x) != cudaSuccess) return ACE_E_CUDA; \
  } while (0)

// Small device headers (status words, counts) come back to the host through
// pinned, mapped host memory written by a one-warp kernel, not through a
// copy: a copy would queue on the copy engines behind large transfers that
// other streams have in flight.  The library's only allocation, 256 KiB of
// host memory, is made once per process; calls take 256-byte slots in turn
// and hold one only while they wait for their stream.
constexpr uint32_t kMirrorSlots = 1024, kMirrorBytes = 256;

__global__ void mirror_kernel(const uint32_t* src, uint32_t* dst, uint32_t words) {
  for (uint32_t i = threadIdx.x; i < words; i += blockDim.x) dst[i] = *(volatile const uint32_t*)(src + i);
}

std::once_flag g_mirror_once;
uint8_t* g_mirror_host = nullptr;
uint8_t* g_mirror_dev = nullptr;
std::atomic<uint32_t> g_mirror_next{0};

// Reads bytes (a multiple of 4, at most 256) at d_src into h_dst after the
// work already on s; synchronises s.
ace_status read_header(const void* d_src, void* h_dst, uint32_t bytes, cudaStream_t s) {
  std::call_once(g_mirror_once, [] {
    void* h = nullptr;
    void* d = nullptr;
    if (cudaHostAlloc(&h, (size_t)kMirrorSlots * kMirrorBytes, cudaHostAllocMapped | cudaHostAllocPortable) !=
        cudaSuccess)
      return;
    if (cudaHostGetDevicePointer(&d, h, 0) != cudaSuccess) {
      cudaFreeHost(h);
      return;
    }
    g_mirror_host = static_cast<uint8_t*>(h);
    g_mirror_dev = static_cast<uint8_t*>(d);
  });
  if (!g_mirror_host || bytes > kMirrorBytes || (bytes & 3)) return ACE_E_CUDA;
  const uint32_t k = g_mirror_next.fetch_add(1) % kMirrorSlots;
  mirror_kernel<<<1, 64, 0, s>>>(static_cast<const uint32_t*>(d_src),
                                 reinterpret_cast<uint32_t*>(g_mirror_dev + (size_t)k * kMirrorBytes), bytes / 4);
  CUDA_TRY(cudaGetLastError());
  CUDA_TRY(cudaStreamSynchronize(s));
  std::memcpy(h_dst, (const void*)(g_mirror_host + (size_t)k * kMirrorBytes), bytes);
  return ACE_OK;
}

// Launch shape of one three-pass decode: per pass the shared memory of a warp
// (tokens: tables, two rings and escape values; literals: tables, a ring and
// the token window; matches: the match records) and the grid.
struct Launch {
  uint32_t warps, chunk;
  uint32_t smem[4];  // [PASS_FUSED]: the largest of the three (its phases reuse one area)
  uint32_t grid[4];
  uint64_t timeout;
  uint32_t schedule;
  uint32_t long_min;  // the copy-width knob as the long class's shortest match
};

template <class K>
ace_status occupancy(K kernel, int device, uint32_t warps, size_t smem, int* occ) {
  int optin = 0;
  CUDA_TRY(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device));
  cudaFuncAttributes fa;
  CUDA_TRY(cudaFuncGetAttributes(&fa, kernel));
  const size_t dyn_max = (size_t)optin - fa.sharedSizeBytes;  // the kernel's static shared memory counts too
  if (smem > dyn_max) {
    *occ = -1;  // this many warps with this much shared memory do not fit one CTA
    return ACE_OK;
  }
  // allow every configuration up to the opt-in limit, so launches planned
  // earlier with other shapes stay valid
  CUDA_TRY(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn_max));
  int o = 0;
  CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, kernel, 32 * warps, smem));
  *occ = o > 0 ? o : -1;
  return ACE_OK;
}

// occ_cache: 4 x 9 x 9 ints (pass, warps per CTA, window / 32), 0 = unknown;
// k3 is the fused pass
template <class K0, class K1, class K2, class K3>
ace_status plan_launch(const ace_index* idx, const ace_tune* tune, uint32_t log2B, uint64_t max_items,
                       K0 k0, K1 k1, K2 k2, K3 k3, int* occ_cache, Launch* L,
                       uint32_t lit_ring = kRing) {
  ace_tune t = tune ? *tune : idx->tune;
  L->warps = t.warps_per_cta ? t.warps_per_cta : 4;
  L->chunk = t.chunk_tokens ? t.chunk_tokens : 128;
  if (L->warps > kMaxWarpsPerCta || (L->chunk & 31) || L->chunk > kMaxWindow) return ACE_E_INVAL;
  L->timeout = t.wait_timeout_ns ? t.wait_timeout_ns : kDefaultTimeoutNs;
  L->schedule = t.schedule;
  if (L->schedule > ACE_SCHEDULE_FUSED) return ACE_E_INVAL;
  if (t.copy_width != 0 && t.copy_width != 8 && t.copy_width != 16) return ACE_E_INVAL;
  // the library's choice (0): 16-byte pieces from 33 bytes (genome 1 GiB
  // 1.37 ms against 1.43; FASTQ and text unchanged)
  L->long_min = t.copy_width == 8 ? kLongMinNarrow : kLongMinWide;
  // automatic: the pass schedule, measured faster on every profile (the
  // fused launch's match jobs of the first levels form a serial chain)
  if (L->schedule == ACE_SCHEDULE_AUTO) L->schedule = ACE_SCHEDULE_PASSES;
  L->smem[PASS_TOKENS] = tok_smem_bytes(esc_cap(log2B));
  L->smem[PASS_LITERALS] = lit_smem_bytes(L->chunk, lit_ring);
  L->smem[PASS_MATCH] = kMatchSmem;
  L->smem[PASS_FUSED] = std::max(std::max(L->smem[PASS_TOKENS], L->smem[PASS_LITERALS]), L->smem[PASS_MATCH]);
  int per[4];
  for (int p = 0; p < 4; p++) {
    int& c = occ_cache[(p * 9 + L->warps) * 9 + L->chunk / 32];
    if (c == 0) {
      const size_t smem = (size_t)L->warps * L->smem[p];
      ace_status rc = p == 0   ? occupancy(k0, idx->device, L->warps, smem, &c)
                      : p == 1 ? occupancy(k1, idx->device, L->warps, smem, &c)
                      : p == 2 ? occupancy(k2, idx->device, L->warps, smem, &c)
                               : occupancy(k3, idx->device, L->warps, smem, &c);
      if (rc) return rc;
    }
    if (c < 0) return ACE_E_INVAL;
    per[p] = c;
    if (t.ctas_per_sm && (int)t.ctas_per_sm < per[p]) per[p] = (int)t.ctas_per_sm;
  }
  uint64_t need = std::max<uint64_t>(1, (max_items + L->warps - 1) / L->warps);
  for (int p = 0; p < 4; p++) L->grid[p] = (uint32_t)std::min<uint64_t>((uint64_t)idx->num_sms * per[p], need);
  return ACE_OK;
}

template <bool SEEK>
ace_status plan_index_launch(const ace_index* idx, const ace_tune* tune, uint64_t max_items, Launch* L) {
  return plan_launch(idx, tune, idx->h.log2_block, max_items, decode_kernel<SEEK, PASS_TOKENS>,
                     decode_kernel<SEEK, PASS_LITERALS>, decode_kernel<SEEK, PASS_MATCH>,
                     decode_kernel<SEEK, PASS_FUSED>, &idx->occ_cache[SEEK][0][0][0], L,
                     SEEK ? kSeekRing : kRing);
}

// Launches the passes in the mask (bit p: pass p) in order on s, each with
// its own shared memory per warp.
template <class K0, class K1, class K2, class Args>
void launch_passes(const Launch& L, uint32_t passes, K0 k0, K1 k1, K2 k2, Args a, cudaStream_t s) {
  const uint32_t th = 32 * L.warps;
  if (passes & 1) {
    a.warp_smem = L.smem[0];
    k0<<<L.grid[0], th, (size_t)L.warps * L.smem[0], s>>>(a);
  }
  if (passes & 2) {
    a.warp_smem = L.smem[1];
    k1<<<L.grid[1], th, (size_t)L.warps * L.smem[1], s>>>(a);
  }
  if (passes & 4) {
    a.warp_smem = L.smem[2];
    k2<<<L.grid[2], th, (size_t)L.warps * L.smem[2], s>>>(a);
  }
}

// The fused pass: one launch for the whole decode.
template <class K3, class Args>
void launch_fused(const Launch& L, K3 k3, Args a, cudaStream_t s) {
  a.warp_smem = L.smem[PASS_FUSED];
  k3<<<L.grid[PASS_FUSED], 32 * L.warps, (size_t)L.warps * L.smem[PASS_FUSED], s>>>(a);
}

template <bool SEEK>
void launch_three_pass(const Launch& L, const DecodeArgs& a, cudaStream_t s) {
  launch_passes(L, 7, decode_kernel<SEEK, PASS_TOKENS>, decode_kernel<SEEK, PASS_LITERALS>,
                decode_kernel<SEEK, PASS_MATCH>, a, s);
}

// A seek after its closure kernel, over the level-ordered work list: by
// default one fused launch (each warp decodes a block through both layers,
// waiting, bounded, only on pending members of the closure); with the pass
// schedule, tokens and literals over the list, then one match launch that
// waits the same way.  (One launch per level, as whole decodes by passes do,
// is slower for a seek's hundred-odd blocks.)
ace_status launch_seek(const ace_index* idx, const Launch& L, const DecodeArgs& a, cudaStream_t s) {
  (void)idx;
  if (L.schedule == ACE_SCHEDULE_FUSED) launch_fused(L, decode_kernel<true, PASS_FUSED>, a, s);
  else launch_three_pass<true>(L, a, s);
  return ACE_OK;
}

}  // namespace

extern "C" {

const char* ace_status_str(ace_status s) {
  switch (s) {
    case ACE_OK: return "ACE_OK";
    case ACE_E_INVAL: return "ACE_E_INVAL";
    case ACE_E_CORRUPT: return "ACE_E_CORRUPT";
    case ACE_E_RANGE: return "ACE_E_RANGE";
    case ACE_E_NOMEM: return "ACE_E_NOMEM";
    case ACE_E_TIMEOUT: return "ACE_E_TIMEOUT";
    case ACE_E_CUDA: return "ACE_E_CUDA";
    default: return "ACE_E_UNKNOWN";
  }
}

ace_status ace_index_size(const void* h_header, uint64_t header_bytes, uint64_t* index_bytes) {
  if (!index_bytes) return ACE_E_INVAL;
  ace_file_header h;
  ace_status rc = parse_header(h_header, header_bytes, &h);
  if (rc) return rc;
  *index_bytes = index_layout(h.n_blocks).total;
  return ACE_OK;
}

}  // extern "C"

namespace {

// A new host handle over the archive and index memory, and the arguments of
// the index kernels.  Returns null with *rc set on failure.
ace_index* index_handle(const void* d_archive, uint64_t archive_bytes, const void* h_header, uint64_t header_bytes,
                        void* d_index_mem, uint64_t index_bytes, IndexArgs* a, ace_status* rc) {
  *rc = ACE_E_INVAL;
  if (!d_index_mem || (!d_archive && archive_bytes)) return nullptr;
  if (!aligned(d_archive, 16) || !aligned(d_index_mem, 256)) return nullptr;
  ace_file_header h;
  *rc = parse_header(h_header, header_bytes, &h);
  if (*rc) return nullptr;
  *rc = ACE_E_CORRUPT;
  if (h.archive_bytes > archive_bytes) return nullptr;
  IndexLayout L = index_layout(h.n_blocks);
  *rc = ACE_E_NOMEM;
  if (index_bytes < L.total) return nullptr;
  ace_index* idx = new (std::nothrow) ace_index();
  if (!idx) return nullptr;
  idx->d_arc = static_cast<const uint8_t*>(d_archive);
  idx->arc_bytes = archive_bytes;
  idx->h = h;
  idx->d_mem = static_cast<uint8_t*>(d_index_mem);
  idx->mem_bytes = index_bytes;
  idx->d_ih = reinterpret_cast<IndexHdr*>(idx->d_mem);
  idx->d_level = reinterpret_cast<uint32_t*>(idx->d_mem + L.level);
  idx->d_order = reinterpret_cast<uint32_t*>(idx->d_mem + L.order);
  idx->d_dep_ptr = reinterpret_cast<const uint32_t*>(idx->d_arc + h.deps_off);
  idx->tune = ace_tune{};
  *rc = ACE_E_CUDA;
  if (cudaGetDevice(&idx->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&idx->num_sms, cudaDevAttrMultiProcessorCount, idx->device) != cudaSuccess) {
    delete idx;
    return nullptr;
  }
  // the interval table's bounds are checked on the device with the rest
  idx->d_dep_iv = reinterpret_cast<const uint32_t*>(idx->d_arc + h.deps_off + 4 * (h.n_blocks + 1));
  a->arc = idx->d_arc;
  a->dir = reinterpret_cast<const ace_block_dir*>(idx->d_arc + h.dir_off);
  a->dep_ptr = idx->d_dep_ptr;
  a->dep_iv = idx->d_dep_iv;
  a->ih = idx->d_ih;
  a->level = idx->d_level;
  a->order = idx->d_order;
  a->lv_count = reinterpret_cast<uint32_t*>(idx->d_mem + L.lv_count);
  a->lv_cursor = reinterpret_cast<uint32_t*>(idx->d_mem + L.lv_cursor);
  a->match_ptr = reinterpret_cast<uint64_t*>(idx->d_mem + L.match_ptr);
  idx->d_match_ptr = a->match_ptr;
  idx->d_lv_count = a->lv_count;
  a->nb = h.n_blocks;
  a->total = h.total_size;
  a->payload_off = h.payload_off;
  a->arc_bytes = h.archive_bytes;
  a->deps_off = h.deps_off;
  a->max_iv = (h.payload_off - h.deps_off - 4 * (h.n_blocks + 1)) / 8;
  a->log2B = h.log2_block;
  a->w = h.off_width;
  *rc = ACE_OK;
  return idx;
}

// The handle's copies of what the index header holds.
ace_status index_adopt(ace_index* idx, const IndexHdr& ih) {
  if (ih.status) return (ace_status)ih.status;
  idx->n_iv = ih.n_iv;
  idx->max_ntok = ih.max_ntok;
  idx->n_levels = ih.n_levels;
  idx->n_matches = ih.n_matches;
  idx->by_levels = ih.n_levels <= kMaxLevelLaunches;
  if (idx->by_levels) {
    idx->level_start[0] = 0;
    for (uint32_t l = 0; l < ih.n_levels; l++) idx->level_start[l + 1] = idx->level_start[l] + ih.lvc[l];
    if (idx->level_start[ih.n_levels] != idx->h.n_blocks) return ACE_E_CORRUPT;
  }
  return ACE_OK;
}

// FNV-1a 64 of host bytes (the stored index's checksum).
uint64_t host_fnv1a64(const uint8_t* p, uint64_t n) {
  uint64_t h = 0xcbf29ce484222325ull;
  for (uint64_t i = 0; i < n; i++) {
    h ^= p[i];
    h *= 0x100000001b3ull;
  }
  return h;
}

// Header of a stored index: the archive header it belongs to, the index
// memory's size and checksum; the index memory follows.
struct IndexBlobHdr {
  uint32_t magic;  // "ACEI"
  uint32_t version;
  ace_file_header arc;
  uint64_t index_bytes;
  uint64_t fnv;
  uint8_t pad[168];
};
static_assert(sizeof(IndexBlobHdr) == 256, "stored index header");
constexpr uint32_t kIndexMagic = 0x49454341u;  // "ACEI"

}  // namespace

extern "C" {

ace_status ace_index_build(const void* d_archive, uint64_t archive_bytes, const void* h_header,
                           uint64_t header_bytes, void* d_index_mem, uint64_t index_bytes, cudaStream_t s,
                           ace_index** out) {
  if (!out) return ACE_E_INVAL;
  IndexArgs a;
  ace_status rc;
  ace_index* idx = index_handle(d_archive, archive_bytes, h_header, header_bytes, d_index_mem, index_bytes, &a, &rc);
  if (!idx) return rc;
  auto bail = [&](ace_status r) {
    delete idx;
    return r;
  };
  const ace_file_header& h = idx->h;
  if (cudaMemsetAsync(idx->d_mem, 0, index_layout(h.n_blocks).total, s) != cudaSuccess) return bail(ACE_E_CUDA);
  if (h.n_blocks) {
    // every step on the device, each skipping once the header holds an
    // error; the host reads the header once at the end
    uint32_t g = (uint32_t)((h.n_blocks + 255) / 256);
    validate_kernel<<<g, 256, 0, s>>>(a);
    match_scan_kernel<<<1, 1024, 0, s>>>(a);
    const uint32_t gs = (uint32_t)std::min<uint64_t>((h.n_blocks + 7) / 8, (uint64_t)idx->num_sms * 8);
    for (uint32_t k = 0; k < kLevelSweeps; k++) levels_sweep_kernel<<<gs, 256, 0, s>>>(a, k);
    levels_kernel<<<1, 1024, 0, s>>>(a);
    level_hist_kernel<<<g, 256, 0, s>>>(a);
    level_scan_kernel<<<1, 1024, 0, s>>>(a);
    level_scatter_kernel<<<g, 256, 0, s>>>(a);
    IndexHdr ih;
    if (read_header(idx->d_ih, &ih, sizeof ih, s) != ACE_OK) return bail(ACE_E_CUDA);
    rc = index_adopt(idx, ih);
    if (rc) return bail(rc);
  }
  *out = idx;
  return ACE_OK;
}

ace_status ace_index_export_size(const ace_index* idx, uint64_t* bytes) {
  if (!idx || !bytes) return ACE_E_INVAL;
  *bytes = sizeof(IndexBlobHdr) + index_layout(idx->h.n_blocks).total;
  return ACE_OK;
}

ace_status ace_index_export(const ace_index* idx, void* h_blob, uint64_t blob_bytes, cudaStream_t s) {
  if (!idx || !h_blob) return ACE_E_INVAL;
  const uint64_t n = index_layout(idx->h.n_blocks).total;
  if (blob_bytes < sizeof(IndexBlobHdr) + n) return ACE_E_NOMEM;
  uint8_t* p = static_cast<uint8_t*>(h_blob);
  CUDA_TRY(cudaMemcpyAsync(p + sizeof(IndexBlobHdr), idx->d_mem, n, cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  IndexBlobHdr bh{};
  bh.magic = kIndexMagic;
  bh.version = 1;
  bh.arc = idx->h;
  bh.index_bytes = n;
  bh.fnv = host_fnv1a64(p + sizeof(IndexBlobHdr), n);
  std::memcpy(p, &bh, sizeof bh);
  return ACE_OK;
}

ace_status ace_index_import(const void* d_archive, uint64_t archive_bytes, const void* h_header, uint64_t header_bytes,
                            const void* h_blob, uint64_t blob_bytes, void* d_index_mem, uint64_t index_bytes,
                            cudaStream_t s, ace_index** out) {
  if (!out || !h_blob || blob_bytes < sizeof(IndexBlobHdr)) return ACE_E_INVAL;
  IndexArgs a;
  ace_status rc;
  ace_index* idx = index_handle(d_archive, archive_bytes, h_header, header_bytes, d_index_mem, index_bytes, &a, &rc);
  if (!idx) return rc;
  auto bail = [&](ace_status r) {
    delete idx;
    return r;
  };
  const ace_file_header& h = idx->h;
  const uint64_t n = index_layout(h.n_blocks).total;
  IndexBlobHdr bh;
  std::memcpy(&bh, h_blob, sizeof bh);
  const uint8_t* body = static_cast<const uint8_t*>(h_blob) + sizeof(IndexBlobHdr);
  // the stored index must belong to this archive and arrive whole
  if (bh.magic != kIndexMagic || bh.version != 1 || std::memcmp(&bh.arc, &h, sizeof h) != 0 || bh.index_bytes != n ||
      blob_bytes < sizeof(IndexBlobHdr) + n || host_fnv1a64(body, n) != bh.fnv)
    return bail(ACE_E_CORRUPT);
  if (cudaMemcpyAsync(idx->d_mem, body, n, cudaMemcpyHostToDevice, s) != cudaSuccess) return bail(ACE_E_CUDA);
  if (h.n_blocks) {
    // the archive is checked as at a build (directory, dependency table,
    // match counts, largest token count: recomputed over the stored values),
    // then the stored levels and order against it
    IndexLayout L = index_layout(h.n_blocks);
    if (cudaMemsetAsync(idx->d_mem, 0, 12, s) != cudaSuccess) return bail(ACE_E_CUDA);  // status words
    uint32_t g = (uint32_t)((h.n_blocks + 255) / 256);
    validate_kernel<<<g, 256, 0, s>>>(a);
    match_scan_kernel<<<1, 1024, 0, s>>>(a);
    const uint32_t gs = (uint32_t)std::min<uint64_t>((h.n_blocks + 7) / 8, (uint64_t)idx->num_sms * 8);
    level_verify_kernel<<<gs, 256, 0, s>>>(a);
    uint32_t* seen = reinterpret_cast<uint32_t*>(idx->d_mem + L.seen);
    if (cudaMemsetAsync(seen, 0, 4 * h.n_blocks, s) != cudaSuccess) return bail(ACE_E_CUDA);
    order_verify_kernel<<<g, 256, 0, s>>>(a, seen);
    IndexHdr ih;
    if (read_header(idx->d_ih, &ih, sizeof ih, s) != ACE_OK) return bail(ACE_E_CUDA);
    rc = index_adopt(idx, ih);
    if (rc) return bail(rc);
  }
  *out = idx;
  return ACE_OK;
}

ace_status ace_index_info(const ace_index* idx, ace_info* info) {
  if (!idx || !info) return ACE_E_INVAL;
  info->total_size = idx->h.total_size;
  info->n_blocks = idx->h.n_blocks;
  info->archive_bytes = idx->h.archive_bytes;
  info->n_dep_intervals = idx->n_iv;
  info->block_size = 1u << idx->h.log2_block;
  info->off_width = idx->h.off_width;
  info->n_levels = idx->n_levels;
  info->reserved = 0;
  return ACE_OK;
}

ace_status ace_index_levels(const ace_index* idx, uint32_t* h_counts, uint32_t n, cudaStream_t s) {
  if (!idx || (!h_counts && n)) return ACE_E_INVAL;
  const uint32_t m = std::min(n, idx->n_levels);
  if (!m) return ACE_OK;
  if (idx->by_levels) {
    for (uint32_t l = 0; l < m; l++) h_counts[l] = idx->level_start[l + 1] - idx->level_start[l];
    return ACE_OK;
  }
  const IndexLayout L = index_layout(idx->h.n_blocks);
  CUDA_TRY(cudaMemcpyAsync(h_counts, idx->d_mem + L.lv_count, 4ull * m, cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  return ACE_OK;
}

ace_status ace_index_set_tune(ace_index* idx, const ace_tune* tune) {
  if (!idx) return ACE_E_INVAL;
  if (tune && (tune->warps_per_cta > kMaxWarpsPerCta || (tune->chunk_tokens & 31) || tune->chunk_tokens > kMaxWindow ||
               tune->schedule > ACE_SCHEDULE_FUSED ||
               (tune->copy_width != 0 && tune->copy_width != 8 && tune->copy_width != 16)))
    return ACE_E_INVAL;
  idx->tune = tune ? *tune : ace_tune{};
  return ACE_OK;
}

ace_status ace_index_free(ace_index* idx) {
  delete idx;
  return ACE_OK;
}

ace_status ace_scratch_size(const ace_index* idx, uint64_t max_seek_blocks, uint64_t* bytes) {
  if (!idx || !bytes) return ACE_E_INVAL;
  *bytes = scratch_layout(idx->h.n_blocks, idx->h.log2_block, max_seek_blocks, idx->max_ntok, idx->n_matches).total;
  return ACE_OK;
}

ace_status ace_scratch_init(const ace_index* idx, void* d_scratch, uint64_t scratch_bytes, cudaStream_t s) {
  if (!idx || !d_scratch || !aligned(d_scratch, 256)) return ACE_E_INVAL;
  ScratchLayout L0 = scratch_layout(idx->h.n_blocks, idx->h.log2_block, 0, idx->max_ntok, idx->n_matches);
  if (scratch_bytes < L0.total) return ACE_E_NOMEM;
  // header, ready flags, and (when present) slot map, work list and marks
  uint64_t clear = L0.tail;
  CUDA_TRY(cudaMemsetAsync(d_scratch, 0, clear, s));
  return ACE_OK;
}

}  // extern "C"

namespace {

// passes: bit 0 the token pass (with the call's header reset before it),
// bit 1 the literal pass, bit 2 the match pass.
ace_status decode_all_passes(const ace_index* idx, uint32_t passes, void* d_out, uint64_t out_bytes, void* d_scratch,
                             uint64_t scratch_bytes, const ace_tune* tune, cudaStream_t s) {
  if (!idx || !d_scratch || (!d_out && idx->h.total_size)) return ACE_E_INVAL;
  if (!aligned(d_scratch, 256) || !aligned(d_out, 16)) return ACE_E_INVAL;
  if (out_bytes < idx->h.total_size) return ACE_E_NOMEM;
  ScratchLayout SL = scratch_layout(idx->h.n_blocks, idx->h.log2_block, 0, idx->max_ntok, idx->n_matches);
  if (scratch_bytes < SL.total) return ACE_E_NOMEM;
  if (!idx->h.n_blocks) return ACE_OK;
  Launch L;
  ace_status rc = plan_index_launch<false>(idx, tune, idx->h.n_blocks, &L);
  if (rc) return rc;
  ScratchHdr* sh = static_cast<ScratchHdr*>(d_scratch);
  DecodeArgs a{};
  a.arc = idx->d_arc;
  a.dir = reinterpret_cast<const ace_block_dir*>(idx->d_arc + idx->h.dir_off);
  a.payload_off = idx->h.payload_off;
  a.total = idx->h.total_size;
  a.nb = idx->h.n_blocks;
  a.log2B = idx->h.log2_block;
  a.w = idx->h.off_width;
  a.window = L.chunk;
  a.max_ntok = idx->max_ntok;
  a.esc_cap = esc_cap(a.log2B);
  a.warp_smem = L.smem[PASS_TOKENS];
  a.n_items = (uint32_t)idx->h.n_blocks;
  a.items = idx->d_order;
  a.out = static_cast<uint8_t*>(d_out);
  a.sh = sh;
  a.ready = reinterpret_cast<uint32_t*>(static_cast<uint8_t*>(d_scratch) + SL.ready);
  a.timeout_ns = L.timeout;
  a.recs = reinterpret_cast<MatchRec*>(static_cast<uint8_t*>(d_scratch) + SL.tail);
  a.match_ptr = idx->d_match_ptr;
  a.level = idx->d_level;
  a.long_min = L.long_min;
  if (passes == 7 && L.schedule == ACE_SCHEDULE_FUSED) {
    // one launch over the (level, block) order; the level counters start at 0
    a.lv_done = reinterpret_cast<uint32_t*>(static_cast<uint8_t*>(d_scratch) + SL.lv_done);
    a.lv_count = idx->d_lv_count;
    CUDA_TRY(cudaMemsetAsync(a.lv_done, 0, 4ull * idx->n_levels, s));
    begin_call_kernel<<<1, 1, 0, s>>>(sh);
    launch_fused(L, decode_kernel<false, PASS_FUSED>, a, s);
    CUDA_TRY(cudaGetLastError());
    return ACE_OK;
  }
  if (passes & 1) begin_call_kernel<<<1, 1, 0, s>>>(sh);
  launch_passes(L, passes & (idx->by_levels ? 3u : 7u), decode_kernel<false, PASS_TOKENS>,
                decode_kernel<false, PASS_LITERALS>, decode_kernel<false, PASS_MATCH>, a, s);
  if ((passes & 4) && idx->by_levels) {
    a.warp_smem = L.smem[PASS_MATCH];
    int& occ = idx->occ_level[L.warps][L.chunk / 32];
    if (occ == 0) {
      rc = occupancy(match_level_kernel, idx->device, L.warps, (size_t)L.warps * L.smem[PASS_MATCH], &occ);
      if (rc) return rc;
    }
    if (occ < 0) return ACE_E_INVAL;
    uint32_t per_sm = (uint32_t)occ;
    const ace_tune t = tune ? *tune : idx->tune;
    if (t.ctas_per_sm && t.ctas_per_sm < per_sm) per_sm = t.ctas_per_sm;
    // levels of at most two blocks per SM: a CTA per block (match_small_kernel)
    const bool small_ok = idx->h.log2_block <= kSmallMaxLog2B;
    const size_t small_smem = small_smem_bytes(idx->h.log2_block);
    if (small_ok && small_smem > 48 * 1024 && !idx->small_attr) {  // one value for every block size
      CUDA_TRY(cudaFuncSetAttribute(match_small_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)small_smem_bytes(kSmallMaxLog2B)));
      idx->small_attr = true;
    }
    for (uint32_t l = 0; l < idx->n_levels; l++) {
      const uint32_t n = idx->level_start[l + 1] - idx->level_start[l];
      if (!n) continue;
      a.items = idx->d_order + idx->level_start[l];
      a.n_items = n;
      a.cur_level = l;
      if (small_ok && n <= 2 * idx->num_sms) {
        match_small_kernel<<<n, kSmallThreads, small_smem, s>>>(a);
        continue;
      }
      const uint32_t grid = (uint32_t)std::min<uint64_t>((uint64_t)idx->num_sms * per_sm, (n + L.warps - 1) / L.warps);
      match_level_kernel<<<grid, 32 * L.warps, (size_t)L.warps * L.smem[PASS_MATCH], s>>>(a);
    }
  }
  CUDA_TRY(cudaGetLastError());
  return ACE_OK;
}

}  // namespace

extern "C" {

ace_status ace_decode_all(const ace_index* idx, void* d_out, uint64_t out_bytes, void* d_scratch,
                          uint64_t scratch_bytes, const ace_tune* tune, cudaStream_t s) {
  return decode_all_passes(idx, 7, d_out, out_bytes, d_scratch, scratch_bytes, tune, s);
}

ace_status ace_decode_pass(const ace_index* idx, int pass, void* d_out, uint64_t out_bytes, void* d_scratch,
                           uint64_t scratch_bytes, const ace_tune* tune, cudaStream_t s) {
  if (pass != ACE_PASS_TOKENS && pass != ACE_PASS_LITERALS && pass != ACE_PASS_MATCH) return ACE_E_INVAL;
  return decode_all_passes(idx, 1u << pass, d_out, out_bytes, d_scratch, scratch_bytes, tune, s);
}

ace_status ace_seek(const ace_index* idx, uint64_t coord, uint64_t len, void* d_out, uint64_t out_bytes,
                    void* d_scratch, uint64_t scratch_bytes, cudaStream_t s) {
  if (!idx || !d_out || !d_scratch || !aligned(d_scratch, 256)) return ACE_E_INVAL;
  if (len == 0 || coord >= idx->h.total_size || len > idx->h.total_size - coord) return ACE_E_RANGE;
  if (out_bytes < len) return ACE_E_NOMEM;
  uint64_t nb = idx->h.n_blocks;
  uint32_t log2B = idx->h.log2_block;
  ScratchLayout S1 = scratch_layout(nb, log2B, 1, idx->max_ntok, 0);
  if (scratch_bytes < S1.total) return ACE_E_NOMEM;
  // the layout before the slots does not depend on the slot count (a seek
  // never decodes more than n_blocks blocks)
  uint64_t cap = std::min<uint64_t>(nb, (scratch_bytes - S1.tail) / slot_bytes(log2B, idx->max_ntok));
  uint64_t first = coord >> log2B, last = (coord + len - 1) >> log2B;
  if (last - first + 1 > cap) return ACE_E_NOMEM;
  uint8_t* base = static_cast<uint8_t*>(d_scratch);
  ScratchHdr* sh = reinterpret_cast<ScratchHdr*>(base);
  ClosureArgs c;
  c.dep_ptr = idx->d_dep_ptr;
  c.dep_iv = idx->d_dep_iv;
  c.sh = sh;
  c.marks = reinterpret_cast<uint32_t*>(base + S1.marks);
  c.front0 = reinterpret_cast<uint32_t*>(base + S1.front0);
  c.front1 = reinterpret_cast<uint32_t*>(base + S1.front1);
  c.work = reinterpret_cast<uint32_t*>(base + S1.work);
  c.slot_of = reinterpret_cast<uint32_t*>(base + S1.slot_of);
  c.nb = nb;
  c.first = first;
  c.last = last;
  c.cap = cap;
  c.level = idx->by_levels ? idx->d_level : nullptr;
  c.n_levels = idx->n_levels;
  c.ready = reinterpret_cast<uint32_t*>(base + S1.ready);
  Launch L;
  ace_status rc = plan_index_launch<true>(idx, nullptr, cap, &L);
  if (rc) return rc;
  // the fused schedule needs the closure's work list in level order
  if (!idx->by_levels) L.schedule = ACE_SCHEDULE_PASSES;
  c.lv_done = L.schedule == ACE_SCHEDULE_FUSED ? reinterpret_cast<uint32_t*>(base + S1.lv_done) : nullptr;
  closure_kernel<<<1, 1024, 0, s>>>(c);
  DecodeArgs a{};
  a.arc = idx->d_arc;
  a.dir = reinterpret_cast<const ace_block_dir*>(idx->d_arc + idx->h.dir_off);
  a.payload_off = idx->h.payload_off;
  a.total = idx->h.total_size;
  a.nb = nb;
  a.log2B = log2B;
  a.w = idx->h.off_width;
  a.window = L.chunk;
  a.max_ntok = idx->max_ntok;
  a.esc_cap = esc_cap(log2B);
  a.warp_smem = L.smem[PASS_TOKENS];
  a.items = c.work;
  a.out = base + S1.tail;
  a.sh = sh;
  a.ready = reinterpret_cast<uint32_t*>(base + S1.ready);
  a.slot_of = c.slot_of;
  a.n_slots = (uint32_t)cap;
  a.slice = static_cast<uint8_t*>(d_out);
  a.coord = coord;
  a.len = len;
  a.timeout_ns = L.timeout;
  a.recs = reinterpret_cast<MatchRec*>(base + S1.tail + (cap << log2B));
  a.match_ptr = nullptr;
  a.level = idx->d_level;
  a.closure_flags = true;
  a.long_min = L.long_min;
  a.lv_done = c.lv_done;
  rc = launch_seek(idx, L, a, s);
  if (rc) return rc;
  CUDA_TRY(cudaGetLastError());
  return ACE_OK;
}

ace_status ace_sync(const ace_index* idx, void* d_scratch, cudaStream_t s) {
  if (!idx || !d_scratch) return ACE_E_INVAL;
  ScratchHdr h;
  ace_status rc = read_header(d_scratch, &h, sizeof h, s);
  if (rc) return rc;
  if (h.status) {
    CUDA_TRY(cudaMemsetAsync(d_scratch, 0, 3 * sizeof(uint32_t), s));
    CUDA_TRY(cudaStreamSynchronize(s));
  }
  return (ace_status)h.status;
}

ace_status ace_host_register(void* h_p, uint64_t bytes, uint32_t read_only, void** d_p) {
  if (!h_p || !bytes || !d_p) return ACE_E_INVAL;
  unsigned flags = cudaHostRegisterMapped | cudaHostRegisterPortable;
  int dev = 0, ro = 0;
  CUDA_TRY(cudaGetDevice(&dev));
  // read-only registration where the platform offers it (a hint only)
  if (read_only && cudaDeviceGetAttribute(&ro, cudaDevAttrHostRegisterReadOnlySupported, dev) == cudaSuccess && ro)
    flags |= cudaHostRegisterReadOnly;
  CUDA_TRY(cudaHostRegister(h_p, bytes, flags));
  if (cudaHostGetDevicePointer(d_p, h_p, 0) != cudaSuccess) {
    cudaHostUnregister(h_p);
    return ACE_E_CUDA;
  }
  return ACE_OK;
}

ace_status ace_host_unregister(void* h_p) {
  if (!h_p) return ACE_E_INVAL;
  CUDA_TRY(cudaHostUnregister(h_p));
  return ACE_OK;
}

ace_status ace_fnv1a64(const void* d_p, uint64_t n, uint64_t* d_result, cudaStream_t s) {
  if ((!d_p && n) || !d_result) return ACE_E_INVAL;
  fnv_kernel<<<1, 1, 0, s>>>(static_cast<const uint8_t*>(d_p), n, d_result);
  CUDA_TRY(cudaGetLastError());
  return ACE_OK;
}

ace_status ace_verify(const ace_index* idx, uint64_t coord, uint64_t len, void* d_buf, uint64_t guard_bytes,
                      uint64_t expected, uint32_t canary_seed, void* d_scratch, uint64_t scratch_bytes,
                      ace_verify_report* rep, cudaStream_t s) {
  if (!idx || !d_buf || !d_scratch || !rep) return ACE_E_INVAL;
  if (len == 0 || coord >= idx->h.total_size || len > idx->h.total_size - coord) return ACE_E_RANGE;
  std::memset(rep, 0, sizeof *rep);
  uint8_t* buf = static_cast<uint8_t*>(d_buf);
  uint8_t* slice = buf + guard_bytes;
  ScratchHdr* sh = static_cast<ScratchHdr*>(d_scratch);
  uint32_t poison_seed = canary_seed ^ 0x5bd1e995u;
  auto guards_bad = [&](uint64_t* out_bad) -> ace_status {
    CUDA_TRY(cudaMemsetAsync(&sh->guard_bad, 0, 8, s));
    if (guard_bytes) {
      count_pattern_mismatch_kernel<<<64, 256, 0, s>>>(buf, guard_bytes, canary_seed, &sh->guard_bad);
      count_pattern_mismatch_kernel<<<64, 256, 0, s>>>(slice + len, guard_bytes, canary_seed ^ 0x9e3779b9u,
                                                       &sh->guard_bad);
    }
    CUDA_TRY(cudaMemcpyAsync(out_bad, &sh->guard_bad, 8, cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    return ACE_OK;
  };
  // set up: canaries around, poison inside
  if (guard_bytes) {
    fill_pattern_kernel<<<64, 256, 0, s>>>(buf, guard_bytes, canary_seed);
    fill_pattern_kernel<<<64, 256, 0, s>>>(slice + len, guard_bytes, canary_seed ^ 0x9e3779b9u);
  }
  fill_pattern_kernel<<<256, 256, 0, s>>>(slice, len, poison_seed);
  CUDA_TRY(cudaGetLastError());
  // phase 1: the slice holds none of the original
  fnv_kernel<<<1, 1, 0, s>>>(slice, len, &sh->fnv);
  CUDA_TRY(cudaMemcpyAsync(&rep->fnv_before, &sh->fnv, 8, cudaMemcpyDeviceToHost, s));
  ace_status rc = guards_bad(&rep->guard_bad_before);
  if (rc) return rc;
  rep->phase1_ok = rep->fnv_before != expected;
  // the seek through both layers
  rc = ace_seek(idx, coord, len, slice, len, d_scratch, scratch_bytes, s);
  if (rc) return rc;
  rep->seek_status = ace_sync(idx, d_scratch, s);
  // phase 2: the slice equals the original; phase 3: the guards are untouched
  fnv_kernel<<<1, 1, 0, s>>>(slice, len, &sh->fnv);
  CUDA_TRY(cudaMemcpyAsync(&rep->fnv_after, &sh->fnv, 8, cudaMemcpyDeviceToHost, s));
  rc = guards_bad(&rep->guard_bad_after);
  if (rc) return rc;
  rep->phase2_ok = rep->seek_status == ACE_OK && rep->fnv_after == expected;
  rep->phase3_ok = rep->guard_bad_before == 0 && rep->guard_bad_after == 0;
  return ACE_OK;
}

// ------------------------------------------------------------ batch (host)

struct ace_batch {
  int device;
  uint32_t n;
  uint8_t* d_scratch;
  uint64_t scratch_bytes;
  uint64_t lv_done_off, lv_done_bytes;  // the fused schedule's level counters
  BatchArgs args;
  Launch L;
  int occ[4][9][9];
};

namespace {

struct BatchLayout {
  uint64_t objs, item_start, ready, lv_done, lv_done_bytes, recs, total, max_ntok, items, n_matches;
  uint32_t max_log2B;
};

ace_status batch_layout(const ace_index* const* idx, uint32_t n, BatchLayout* B) {
  if (!idx || n == 0) return ACE_E_INVAL;
  uint64_t ready = 0, items = 0, max_ntok = 0, matches = 0, levels = 0;
  uint32_t max_log2B = 0;
  int dev = idx[0] ? idx[0]->device : -1;
  for (uint32_t i = 0; i < n; i++) {
    if (!idx[i] || idx[i]->device != dev) return ACE_E_INVAL;
    items += idx[i]->h.n_blocks;
    ready += align256(4 * idx[i]->h.n_blocks);
    matches += idx[i]->n_matches;
    levels += idx[i]->n_levels;
    max_ntok = std::max<uint64_t>(max_ntok, idx[i]->max_ntok);
    max_log2B = std::max<uint32_t>(max_log2B, idx[i]->h.log2_block);
  }
  if (items > 0xFFFFFFF0ull) return ACE_E_INVAL;
  uint64_t o = sizeof(ScratchHdr);
  B->objs = o;
  o = align256(o + n * sizeof(ObjDesc));
  B->item_start = o;
  o = align256(o + 4ull * (n + 1));
  B->ready = o;
  o += ready;
  B->lv_done = o;
  B->lv_done_bytes = 4 * levels;
  o = align256(o + 4 * levels);
  B->recs = o;
  o = align256(o + 16 * matches);
  B->total = o;
  B->n_matches = matches;
  B->max_ntok = max_ntok;
  B->items = items;
  B->max_log2B = max_log2B;
  return ACE_OK;
}

}  // namespace

ace_status ace_batch_scratch_size(const ace_index* const* idx, uint32_t n, uint64_t* bytes) {
  if (!bytes) return ACE_E_INVAL;
  BatchLayout B;
  ace_status rc = batch_layout(idx, n, &B);
  if (rc) return rc;
  *bytes = B.total;
  return ACE_OK;
}

ace_status ace_batch_create(const ace_index* const* idx, uint32_t n, void* const* d_outs, const uint64_t* out_bytes,
                            void* d_scratch, uint64_t scratch_bytes, const ace_tune* tune, cudaStream_t s,
                            ace_batch** out) {
  if (!out || !d_outs || !out_bytes || !d_scratch || !aligned(d_scratch, 256)) return ACE_E_INVAL;
  BatchLayout B;
  ace_status rc = batch_layout(idx, n, &B);
  if (rc) return rc;
  if (scratch_bytes < B.total) return ACE_E_NOMEM;
  uint8_t* base = static_cast<uint8_t*>(d_scratch);
  std::vector<ObjDesc> od(n);
  std::vector<uint32_t> start(n + 1);
  uint64_t ready = B.ready, items = 0, recs = B.recs, lvd = B.lv_done;
  for (uint32_t i = 0; i < n; i++) {
    const ace_index* x = idx[i];
    if (out_bytes[i] < x->h.total_size || (!d_outs[i] && x->h.total_size)) return ACE_E_NOMEM;
    if (!aligned(d_outs[i], 16)) return ACE_E_INVAL;
    od[i] = ObjDesc{x->d_arc,
                    reinterpret_cast<const ace_block_dir*>(x->d_arc + x->h.dir_off),
                    x->h.payload_off,
                    x->h.total_size,
                    static_cast<uint8_t*>(d_outs[i]),
                    reinterpret_cast<uint32_t*>(base + ready),
                    x->d_order,
                    x->d_level,
                    reinterpret_cast<MatchRec*>(base + recs),
                    x->d_match_ptr,
                    reinterpret_cast<uint32_t*>(base + lvd),
                    x->d_lv_count,
                    x->h.log2_block,
                    x->h.off_width,
                    (uint32_t)x->h.n_blocks,
                    0};
    start[i] = (uint32_t)items;
    items += x->h.n_blocks;
    ready += align256(4 * x->h.n_blocks);
    recs += 16 * x->n_matches;
    lvd += 4ull * x->n_levels;
  }
  start[n] = (uint32_t)items;
  ace_batch* b = new (std::nothrow) ace_batch();
  if (!b) return ACE_E_NOMEM;
  b->device = idx[0]->device;
  b->n = n;
  b->d_scratch = base;
  b->scratch_bytes = scratch_bytes;
  b->lv_done_off = B.lv_done;
  b->lv_done_bytes = B.lv_done_bytes;
  // the launch shape uses the largest block size's escape table
  rc = plan_launch(idx[0], tune, B.max_log2B, B.items, batch_decode_kernel<PASS_TOKENS>,
                   batch_decode_kernel<PASS_LITERALS>, batch_decode_kernel<PASS_MATCH>,
                   batch_decode_kernel<PASS_FUSED>, &b->occ[0][0][0], &b->L);
  if (rc == ACE_OK &&
      (cudaMemsetAsync(base, 0, B.recs, s) != cudaSuccess ||
       cudaMemcpyAsync(base + B.objs, od.data(), n * sizeof(ObjDesc), cudaMemcpyHostToDevice, s) != cudaSuccess ||
       cudaMemcpyAsync(base + B.item_start, start.data(), 4ull * (n + 1), cudaMemcpyHostToDevice, s) != cudaSuccess ||
       cudaStreamSynchronize(s) != cudaSuccess))
    rc = ACE_E_CUDA;
  if (rc) {
    delete b;
    return rc;
  }
  BatchArgs& a = b->args;
  a.objs = reinterpret_cast<const ObjDesc*>(base + B.objs);
  a.item_start = reinterpret_cast<const uint32_t*>(base + B.item_start);
  a.n_objs = n;
  a.n_items = (uint32_t)B.items;
  a.window = b->L.chunk;
  a.warp_smem = b->L.smem[PASS_TOKENS];
  a.esc_cap = esc_cap(B.max_log2B);
  a.max_ntok = (uint32_t)B.max_ntok;
  a.sh = reinterpret_cast<ScratchHdr*>(base);
  a.timeout_ns = b->L.timeout;
  a.long_min = b->L.long_min;
  *out = b;
  return ACE_OK;
}

ace_status ace_decode_batch(const ace_batch* b, cudaStream_t s) {
  if (!b) return ACE_E_INVAL;
  if (!b->args.n_items) return ACE_OK;
  const Launch& L = b->L;
  if (L.schedule == ACE_SCHEDULE_FUSED && b->lv_done_bytes)
    CUDA_TRY(cudaMemsetAsync(b->d_scratch + b->lv_done_off, 0, b->lv_done_bytes, s));
  begin_call_kernel<<<1, 1, 0, s>>>(b->args.sh);
  if (L.schedule == ACE_SCHEDULE_FUSED)
    launch_fused(L, batch_decode_kernel<PASS_FUSED>, b->args, s);
  else
    launch_passes(L, 7, batch_decode_kernel<PASS_TOKENS>, batch_decode_kernel<PASS_LITERALS>,
                  batch_decode_kernel<PASS_MATCH>, b->args, s);
  CUDA_TRY(cudaGetLastError());
  return ACE_OK;
}

ace_status ace_batch_sync(const ace_batch* b, cudaStream_t s) {
  if (!b) return ACE_E_INVAL;
  ScratchHdr h;
  ace_status rc = read_header(b->d_scratch, &h, sizeof h, s);
  if (rc) return rc;
  if (h.status) {
    CUDA_TRY(cudaMemsetAsync(b->d_scratch, 0, 3 * sizeof(uint32_t), s));
    CUDA_TRY(cudaStreamSynchronize(s));
  }
  return (ace_status)h.status;
}

ace_status ace_batch_launch_shape(const ace_batch* b, uint32_t* grid, uint32_t* warps_per_cta, uint32_t* window) {
  if (!b) return ACE_E_INVAL;
  if (grid) *grid = b->L.grid[PASS_TOKENS];
  if (warps_per_cta) *warps_per_cta = b->L.warps;
  if (window) *window = b->L.chunk;
  return ACE_OK;
}

ace_status ace_batch_free(ace_batch* b) {
  delete b;
  return ACE_OK;
}

// ------------------------------------------------------ seek batches (host)

struct ace_cache {
  int device;
  uint32_t n_arcs, log2B, n_slots, front_cap, max_reqs;
  uint8_t* mem;
  uint64_t bytes;
  CacheArgs args;
  CacheDecodeArgs dargs;
  Launch L;
  uint64_t req_off;  // requests are staged here by ace_seek_batch_host
  uint64_t owner_off;  // per-slot owners, cleared by a reset
  int occ[4][9][9];
};

namespace {

struct CacheLayout {
  uint64_t arcs, minmax, front0, front1, work, taken, owner_arc, owner_blk, ref, use, reqs, slots, recs, total, max_ntok,
      max_work;
};

// Blocks one seek batch may decode at most (work items): 32 per request the
// batch may hold, at least 1024, at most the slots.  Its match records are
// sized by it rather than by the slot count, since only the blocks a batch
// decodes need records, and only while it runs.
inline uint64_t cache_max_work(uint64_t n_slots, uint32_t max_reqs) {
  return std::min<uint64_t>(n_slots, std::max<uint64_t>(1024, 32ull * max_reqs));
}

CacheLayout cache_layout(const ace_index* const* idx, uint32_t n, uint64_t n_slots, uint32_t max_reqs,
                         uint32_t log2B) {
  CacheLayout C;
  uint64_t max_ntok = 0;
  for (uint32_t i = 0; i < n; i++) max_ntok = std::max<uint64_t>(max_ntok, idx[i]->max_ntok);
  const uint64_t mw = cache_max_work(n_slots, max_reqs);
  uint64_t o = sizeof(CacheHdr);
  C.arcs = o;
  o = align256(o + n * sizeof(CacheArc));
  C.minmax = o;
  o = align256(o + 8ull * n);
  C.front0 = o;
  o = align256(o + 8 * mw);
  C.front1 = o;
  o = align256(o + 8 * mw);
  C.work = o;
  o = align256(o + 8 * mw);
  C.taken = o;
  o = align256(o + 4 * mw);
  C.owner_arc = o;
  o = align256(o + 4 * n_slots);
  C.owner_blk = o;
  o = align256(o + 4 * n_slots);
  C.ref = o;
  o = align256(o + 4 * n_slots);
  C.use = o;
  o = align256(o + 4 * n_slots);
  C.reqs = o;
  o = align256(o + sizeof(ace_seek_req) * (uint64_t)max_reqs);
  C.slots = o;
  o = align256(o + (n_slots << log2B));
  C.recs = o;
  o = align256(o + 16 * max_ntok * mw);
  C.total = o;
  C.max_ntok = max_ntok;
  C.max_work = mw;
  return C;
}

ace_status cache_check(const ace_index* const* idx, uint32_t n) {
  if (!idx || n == 0) return ACE_E_INVAL;
  for (uint32_t i = 0; i < n; i++)
    if (!idx[i] || idx[i]->device != idx[0]->device || idx[i]->h.log2_block != idx[0]->h.log2_block)
      return ACE_E_INVAL;  // one device, one block size per cache
  return ACE_OK;
}

}  // namespace

ace_status ace_cache_size(const ace_index* const* idx, uint32_t n, uint64_t n_slots, uint32_t max_reqs,
                          uint64_t* bytes) {
  ace_status rc = cache_check(idx, n);
  if (rc) return rc;
  if (!bytes || n_slots == 0 || n_slots > 0xFFFFFFF0ull || max_reqs == 0) return ACE_E_INVAL;
  *bytes = cache_layout(idx, n, n_slots, max_reqs, idx[0]->h.log2_block).total;
  return ACE_OK;
}

ace_status ace_archive_state_size(const ace_index* idx, uint64_t* bytes) {
  if (!idx || !bytes) return ACE_E_INVAL;
  uint64_t nb = idx->h.n_blocks;
  *bytes = align256(4 * nb) * 3 + align256(4 * ((nb + 31) / 32));  // ready, slot_of, wpos; marks
  return ACE_OK;
}

ace_status ace_cache_create(const ace_index* const* idx, uint32_t n, void* const* d_states, uint64_t n_slots,
                            uint32_t max_reqs, void* d_mem, uint64_t bytes, const ace_tune* tune, cudaStream_t s,
                            ace_cache** out) {
  ace_status rc = cache_check(idx, n);
  if (rc) return rc;
  if (!out || !d_states || !d_mem || !aligned(d_mem, 256) || n_slots == 0 || max_reqs == 0) return ACE_E_INVAL;
  const uint32_t log2B = idx[0]->h.log2_block;
  CacheLayout C = cache_layout(idx, n, n_slots, max_reqs, log2B);
  if (bytes < C.total) return ACE_E_NOMEM;
  uint8_t* base = static_cast<uint8_t*>(d_mem);
  std::vector<CacheArc> arcs(n);
  for (uint32_t i = 0; i < n; i++) {
    const ace_index* x = idx[i];
    if (!d_states[i] || !aligned(d_states[i], 256)) return ACE_E_INVAL;
    uint8_t* st = static_cast<uint8_t*>(d_states[i]);
    uint64_t nb = x->h.n_blocks;
    arcs[i] = CacheArc{x->d_arc,
                       reinterpret_cast<const ace_block_dir*>(x->d_arc + x->h.dir_off),
                       x->h.payload_off,
                       x->h.total_size,
                       x->d_dep_ptr,
                       x->d_dep_iv,
                       reinterpret_cast<uint32_t*>(st),
                       reinterpret_cast<uint32_t*>(st + align256(4 * nb)),
                       reinterpret_cast<uint32_t*>(st + 3 * align256(4 * nb)),
                       reinterpret_cast<uint32_t*>(st + 2 * align256(4 * nb)),
                       (uint32_t)nb,
                       x->h.off_width};
    uint64_t sb = 0;
    ace_archive_state_size(x, &sb);
    if (cudaMemsetAsync(st, 0, sb, s) != cudaSuccess) return ACE_E_CUDA;
  }
  ace_cache* c = new (std::nothrow) ace_cache();
  if (!c) return ACE_E_NOMEM;
  c->device = idx[0]->device;
  c->n_arcs = n;
  c->log2B = log2B;
  c->n_slots = (uint32_t)n_slots;
  c->front_cap = (uint32_t)C.max_work;
  c->max_reqs = max_reqs;
  c->mem = base;
  c->bytes = bytes;
  c->req_off = C.reqs;
  c->owner_off = C.owner_arc;
  // seek batches run the three passes (their work list is in block order,
  // not level order); the fused entry only sizes like the match pass
  rc = plan_launch(idx[0], tune, log2B, C.max_work, cache_decode_kernel<PASS_TOKENS>,
                   cache_decode_kernel<PASS_LITERALS>, cache_decode_kernel<PASS_MATCH>,
                   cache_decode_kernel<PASS_MATCH>, &c->occ[0][0][0], &c->L, kSeekRing);
  // header (epoch 1: no block is cached, since every ready flag starts at 0)
  CacheHdr h{};
  h.epoch = 1;
  // every slot free (owner archive ~0), reference bits and batch serials 0
  if (rc == ACE_OK &&
      (cudaMemcpyAsync(base, &h, sizeof h, cudaMemcpyHostToDevice, s) != cudaSuccess ||
       cudaMemcpyAsync(base + C.arcs, arcs.data(), n * sizeof(CacheArc), cudaMemcpyHostToDevice, s) != cudaSuccess ||
       cudaMemsetAsync(base + C.owner_arc, 0xff, 4 * n_slots, s) != cudaSuccess ||
       cudaMemsetAsync(base + C.ref, 0, C.reqs - C.ref, s) != cudaSuccess ||
       cudaStreamSynchronize(s) != cudaSuccess))
    rc = ACE_E_CUDA;
  if (rc) {
    delete c;
    return rc;
  }
  CacheArgs& a = c->args;
  a.h = reinterpret_cast<CacheHdr*>(base);
  a.arcs = reinterpret_cast<const CacheArc*>(base + C.arcs);
  a.n_arcs = n;
  a.log2B = log2B;
  a.n_slots = (uint32_t)n_slots;
  a.front_cap = (uint32_t)C.max_work;
  a.front0 = reinterpret_cast<uint32_t*>(base + C.front0);
  a.front1 = reinterpret_cast<uint32_t*>(base + C.front1);
  a.work = reinterpret_cast<uint32_t*>(base + C.work);
  a.taken = reinterpret_cast<uint32_t*>(base + C.taken);
  a.owner_arc = reinterpret_cast<uint32_t*>(base + C.owner_arc);
  a.owner_blk = reinterpret_cast<uint32_t*>(base + C.owner_blk);
  a.ref = reinterpret_cast<uint32_t*>(base + C.ref);
  a.use = reinterpret_cast<uint32_t*>(base + C.use);
  a.arc_minmax = reinterpret_cast<uint32_t*>(base + C.minmax);
  a.slots = base + C.slots;
  a.recs = reinterpret_cast<MatchRec*>(base + C.recs);
  a.reqs = nullptr;
  a.n_reqs = 0;
  CacheDecodeArgs& d = c->dargs;
  d.window = c->L.chunk;
  d.warp_smem = c->L.smem[PASS_TOKENS];
  d.esc_cap = esc_cap(log2B);
  d.max_ntok = (uint32_t)C.max_ntok;
  d.timeout_ns = c->L.timeout;
  d.long_min = c->L.long_min;
  *out = c;
  return ACE_OK;
}

ace_status ace_seek_batch(const ace_cache* c, const ace_seek_req* d_reqs, uint32_t n, void* d_pool, uint64_t pool_bytes,
                          cudaStream_t s) {
  if (!c || (!d_reqs && n) || (!d_pool && n)) return ACE_E_INVAL;
  if (n == 0) return ACE_OK;
  (void)pool_bytes;  // request ranges are validated on the host by ace_seek_batch_host
  CacheArgs a = c->args;
  a.reqs = d_reqs;
  a.n_reqs = n;
  cache_closure_kernel<<<1, 1024, 0, s>>>(a);
  CacheDecodeArgs d = c->dargs;
  d.c = a;
  const Launch& L = c->L;
  launch_passes(L, 7, cache_decode_kernel<PASS_TOKENS>, cache_decode_kernel<PASS_LITERALS>,
                cache_decode_kernel<PASS_MATCH>, d, s);
  cache_copy_kernel<<<std::min<uint32_t>(n, 1024), 256, 0, s>>>(a, static_cast<uint8_t*>(d_pool));
  CUDA_TRY(cudaGetLastError());
  return ACE_OK;
}

ace_status ace_seek_batch_host(const ace_cache* c, const ace_seek_req* h_reqs, const uint64_t* h_totals, uint32_t n,
                               void* d_pool, uint64_t pool_bytes, cudaStream_t s) {
  if (!c || (!h_reqs && n)) return ACE_E_INVAL;
  if (n > c->max_reqs) return ACE_E_NOMEM;
  for (uint32_t i = 0; i < n; i++) {
    const ace_seek_req& q = h_reqs[i];
    if (q.archive >= c->n_arcs) return ACE_E_INVAL;
    if (q.len == 0 || (h_totals && (q.coord >= h_totals[q.archive] || q.len > h_totals[q.archive] - q.coord)))
      return ACE_E_RANGE;
    if (q.out_off + q.len > pool_bytes) return ACE_E_NOMEM;
  }
  ace_seek_req* d = reinterpret_cast<ace_seek_req*>(c->mem + c->req_off);
  if (n) CUDA_TRY(cudaMemcpyAsync(d, h_reqs, n * sizeof(ace_seek_req), cudaMemcpyHostToDevice, s));
  return ace_seek_batch(c, d, n, d_pool, pool_bytes, s);
}

ace_status ace_cache_sync(const ace_cache* c, cudaStream_t s) {
  if (!c) return ACE_E_INVAL;
  CacheHdr h;
  ace_status rc = read_header(c->mem, &h, sizeof h, s);
  if (rc) return rc;
  if (h.status) {
    CUDA_TRY(cudaMemsetAsync(c->mem, 0, 3 * sizeof(uint32_t), s));
    CUDA_TRY(cudaStreamSynchronize(s));
  }
  return (ace_status)h.status;
}

ace_status ace_cache_usage(const ace_cache* c, uint32_t* used_slots, uint32_t* n_slots, cudaStream_t s) {
  if (!c) return ACE_E_INVAL;
  CacheHdr h;
  ace_status rc = read_header(c->mem, &h, sizeof h, s);
  if (rc) return rc;
  if (used_slots) *used_slots = h.n_cached;
  if (n_slots) *n_slots = c->n_slots;
  return ACE_OK;
}

ace_status ace_cache_reset(const ace_cache* c, cudaStream_t s) {
  if (!c) return ACE_E_INVAL;
  cache_reset_kernel<<<1, 1, 0, s>>>(c->args.h);
  CUDA_TRY(cudaGetLastError());
  CUDA_TRY(cudaMemsetAsync(c->mem + c->owner_off, 0xff, 4ull * c->n_slots, s));
  return ACE_OK;
}

ace_status ace_cache_counters(const ace_cache* c, uint64_t* h_evicted, uint64_t* h_decoded, cudaStream_t s) {
  if (!c) return ACE_E_INVAL;
  CacheHdr h;
  ace_status rc = read_header(c->mem, &h, sizeof h, s);
  if (rc) return rc;
  if (h_evicted) *h_evicted = h.evicted;
  if (h_decoded) *h_decoded = h.decoded;
  return ACE_OK;
}

ace_status ace_cache_limits(const ace_cache* c, uint32_t* h_n_slots, uint32_t* h_max_work, uint32_t* h_max_reqs) {
  if (!c) return ACE_E_INVAL;
  if (h_n_slots) *h_n_slots = c->n_slots;
  if (h_max_work) *h_max_work = c->front_cap;
  if (h_max_reqs) *h_max_reqs = c->max_reqs;
  return ACE_OK;
}

ace_status ace_cache_free(ace_cache* c) {
  delete c;
  return ACE_OK;
}

// -------------------------------------------------- seek without allocation
//
// Some callers cannot allocate device memory at all: a host application
// that owns every byte of device memory through its own pool, a plug-in
// loaded into such an application, or a latency-critical request thread
// that must never reach the allocator.  ace_seek_noalloc serves them: it
// takes its scratch from a fixed array that lives in this library's device
// image, so the caller passes only the archive's index and the output.
//
// The array is kStaticScratchBytes (32 MiB) on every GPU that loads the
// library, held until the process exits.  It is shared by every call on a
// device and keeps the last call's contents; calls that overlap on the GPU
// race on it and must be ordered by the caller (one stream, or events).

namespace {

constexpr uint64_t kStaticScratchBytes = 32ull << 20;
constexpr int kMaxDevices = 64;

__device__ __align__(256) uint8_t g_static_scratch[kStaticScratchBytes];

std::mutex g_static_mu;
uint8_t* g_static_ptr[kMaxDevices];  // device address of g_static_scratch, per device

// The host-side name g_static_scratch is a stand-in, not a device address:
// the address is looked up once per device, with that device current.
ace_status static_scratch(int device, uint8_t** out) {
  if (device < 0 || device >= kMaxDevices) return ACE_E_INVAL;
  std::lock_guard<std::mutex> lock(g_static_mu);
  if (!g_static_ptr[device]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || !p) return ACE_E_CUDA;
    g_static_ptr[device] = static_cast<uint8_t*>(p);
  }
  *out = g_static_ptr[device];
  return ACE_OK;
}

}  // namespace

ace_status ace_seek_noalloc(const ace_index* idx, uint64_t coord, uint64_t len, void* d_out, uint64_t out_bytes,
                            cudaStream_t s) {
  if (!idx || !d_out) return ACE_E_INVAL;
  if (len == 0 || coord >= idx->h.total_size || len > idx->h.total_size - coord) return ACE_E_RANGE;
  if (out_bytes < len) return ACE_E_NOMEM;
  int cur = -1;
  CUDA_TRY(cudaGetDevice(&cur));
  if (cur != idx->device) return ACE_E_INVAL;  // the index's device must be current
  uint8_t* base = nullptr;
  ace_status rc = static_scratch(cur, &base);
  if (rc) return rc;
  const uint64_t nb = idx->h.n_blocks;
  const uint32_t log2B = idx->h.log2_block;
  ScratchLayout S = scratch_layout(nb, log2B, 1, idx->max_ntok, 0);
  if (S.tail > kStaticScratchBytes) return ACE_E_NOMEM;  // archive too large for the fixed scratch
  uint64_t cap = std::min<uint64_t>(nb, (kStaticScratchBytes - S.tail) / slot_bytes(log2B, idx->max_ntok));
  uint64_t first = coord >> log2B, last = (coord + len - 1) >> log2B;
  if (last - first + 1 > cap) return ACE_E_NOMEM;  // more target blocks than slots
  ScratchHdr* sh = reinterpret_cast<ScratchHdr*>(base);
  // The array may hold what a call on another archive, with another layout,
  // left there.  The closure marks must start clear, and so must the ready
  // flags: a stale word equal to this call's epoch would pass a block outside
  // the closure as a member (epochs are never 0).
  CUDA_TRY(cudaMemsetAsync(base + S.ready, 0, S.slot_of - S.ready, s));
  CUDA_TRY(cudaMemsetAsync(base + S.marks, 0, S.front0 - S.marks, s));
  CUDA_TRY(cudaMemsetAsync(base, 0, 3 * sizeof(uint32_t), s));  // status word
  ClosureArgs c;
  c.dep_ptr = idx->d_dep_ptr;
  c.dep_iv = idx->d_dep_iv;
  c.sh = sh;
  c.marks = reinterpret_cast<uint32_t*>(base + S.marks);
  c.front0 = reinterpret_cast<uint32_t*>(base + S.front0);
  c.front1 = reinterpret_cast<uint32_t*>(base + S.front1);
  c.work = reinterpret_cast<uint32_t*>(base + S.work);
  c.slot_of = reinterpret_cast<uint32_t*>(base + S.slot_of);
  c.nb = nb;
  c.first = first;
  c.last = last;
  c.cap = cap;
  c.level = idx->by_levels ? idx->d_level : nullptr;
  c.n_levels = idx->n_levels;
  c.ready = reinterpret_cast<uint32_t*>(base + S.ready);
  Launch L;
  rc = plan_index_launch<true>(idx, nullptr, cap, &L);
  if (rc) return rc;
  if (!idx->by_levels) L.schedule = ACE_SCHEDULE_PASSES;
  c.lv_done = L.schedule == ACE_SCHEDULE_FUSED ? reinterpret_cast<uint32_t*>(base + S.lv_done) : nullptr;
  closure_kernel<<<1, 1024, 0, s>>>(c);
  DecodeArgs a{};
  a.arc = idx->d_arc;
  a.dir = reinterpret_cast<const ace_block_dir*>(idx->d_arc + idx->h.dir_off);
  a.payload_off = idx->h.payload_off;
  a.total = idx->h.total_size;
  a.nb = nb;
  a.log2B = log2B;
  a.w = idx->h.off_width;
  a.window = L.chunk;
  a.max_ntok = idx->max_ntok;
  a.esc_cap = esc_cap(log2B);
  a.warp_smem = L.smem[PASS_TOKENS];
  a.items = c.work;
  a.out = base + S.tail;
  a.sh = sh;
  a.ready = reinterpret_cast<uint32_t*>(base + S.ready);
  a.slot_of = c.slot_of;
  a.n_slots = (uint32_t)cap;
  a.slice = static_cast<uint8_t*>(d_out);
  a.coord = coord;
  a.len = len;
  a.timeout_ns = L.timeout;
  a.recs = reinterpret_cast<MatchRec*>(base + S.tail + (cap << log2B));
  a.match_ptr = nullptr;
  a.level = idx->d_level;
  a.closure_flags = true;
  a.long_min = L.long_min;
  a.lv_done = c.lv_done;
  rc = launch_seek(idx, L, a, s);
  if (rc) return rc;
  CUDA_TRY(cudaGetLastError());
  // the status lives in the shared array, so the call waits for it
  uint32_t status = 0;
  rc = read_header(base, &status, sizeof status, s);
  if (rc) return rc;
  return (ace_status)status;
}

}  // extern "C"
