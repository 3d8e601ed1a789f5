// state.cuh -- per-vertex state machine of Skipper (Section IV-B, Fig. 4;
// Algorithm 1) on GB300 global memory.
//
// Two layouts of the state array:
//   PackedState<8> (ByteState): one byte per vertex (ACC = 0, RSVD = 1,
//     MCHD = 2 as in Algorithm 1), four vertices packed in a 32-bit word;
//     PackedState<2> (TwoBitState): the same three values in 2 bits, sixteen
//     vertices a word, so the state array is a quarter of the paper's size.
//     Every access is a 32-bit access to the whole word (relaxed loads, 32-bit
//     CAS, 32-bit XOR), so all accesses to a location have the same size and
//     are morally strong in the PTX memory model.  A field CAS is a word CAS
//     that is retried when only a neighbouring field changed.  The holder-only
//     transitions RSVD->MCHD and RSVD->ACC (Algorithm 1 lines 15 and 18, plain
//     stores in the paper) become one atomic XOR on the word, which cannot
//     disturb the neighbouring fields.
//   WordState: one 32-bit word per vertex that doubles as the mate entry:
//     ACC = 0xFFFFFFFF (= unmatched), RSVD = 0xFFFFFFFE, MCHD = the partner id.
//     Claiming v writes u into v's word directly; the holder then stores v into
//     u's word.  No separate mate array is needed.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace skp {

constexpr uint32_t kNone = 0xFFFFFFFFu;
constexpr uint32_t kAcc = 0u, kRsvd = 1u, kMchd = 2u;         // byte states
constexpr uint32_t kWAcc = 0xFFFFFFFFu, kWRsvd = 0xFFFFFFFEu;  // word states
constexpr unsigned kFull = 0xFFFFFFFFu;

// device error word bits
constexpr uint32_t kErrTimeout = 1u;
constexpr uint32_t kErrBadId = 2u;

struct SweepParams {
  uint64_t n;
  uint64_t nnz;
  const int64_t* offsets;
  const uint32_t* nbrs;
  uint32_t* state;      // PackedState: packed words; WordState: == mate
  uint32_t* mate;
  int64_t* part;        // merge-path unit starts: (row, entry) for units+1 diagonals
  uint64_t units;
  uint64_t grain;
  unsigned long long* work;  // next unit to hand out
  uint32_t* err;
  uint64_t spin_limit;
  uint64_t poison;      // vertex + 1 left RESERVED after init (fault injection), 0 = off
  // batched serial mode
  const int64_t* vbase;
  uint64_t num_graphs;
  // statistics (kStats kernels only): see StatSlot
  unsigned long long* stats;
  // 1: the CSR is symmetric; an entry (x, y) with y < x is left to row y
  // (selects the kSym kernel instance)
  uint32_t sym;
  // 1: load only the id quads that hold an entry of a row not known matched
  // (selects the kSel kernel instance; statistics instances load every quad)
  uint32_t sel;
  // 1: stage each 32-row window (row ends and state words) in shared memory
  // with a bulk copy one window ahead (selects the kTile kernel instance)
  uint32_t tile;
  // 1: the plain or symmetric instance compiled for 32 registers a thread
  // (64 warps per SM) instead of 40 (48 warps per SM)
  uint32_t lean;
  // 1: work units handed out in dispersed runs (one run per warp of the grid)
  uint32_t disperse;
};

// Unit order.  Counter value c is unit c (ascending), or, with dispersed
// runs, unit (c mod R) * L + c / R for R runs of L units each, so that the
// units in flight sit at evenly spaced positions and each run is walked in
// order.  Counter values at or past `total` end the walk; values that map
// past the last unit are skipped.
struct UnitOrder {
  uint64_t R, L, units, total;
  __device__ UnitOrder(uint64_t units_, bool disperse, uint64_t runs)
      : R(disperse ? runs : 1), L(disperse ? (units_ + runs - 1) / runs : units_), units(units_),
        total(disperse ? R * L : units_) {}
  __device__ __forceinline__ uint64_t unit(uint64_t c) const { return R == 1 ? c : (c % R) * L + c / R; }
};

// Sweep statistics, kept only by the kStats kernel instances.  A conflict is a
// failed CAS at Algorithm 1 line 11 or 14 (Section VI-E, Table II); a field CAS
// that lost only to a neighbouring field is retried and not counted.
enum StatSlot : int {
  kStEntries = 0,   // neighbour ids read by the sweep
  kStWindows,       // 32-row windows loaded
  kStChunks,        // chunks of up to 128 entries read
  kStAttempts,      // entries that reached Algorithm 1 line 11
  kStMatches,       // successful claims (line 14)
  kStConflicts,     // failed CAS at lines 11 and 14
  kStConflicted,    // entries with at least one conflict
  kStMaxConflicts,  // most conflicts on one entry
  kStHist,          // 10 bins: 1, 2, 3-4, 5-8, 9-16, 17-32, 33-64, 65-128, 129-256, >256
  kStTrans = kStHist + 10,  // state transitions (Fig. 4): ACC->RSVD, ACC->MCHD, RSVD->MCHD, RSVD->ACC
  kStIllegal = kStTrans + 4,  // commits / releases that found the field not RSVD
  kStIdLoads,       // 128-bit id loads issued
  kStIdLoadsOpen,   // of those, quads holding an entry of a row not known matched
  kStCount
};

__device__ __forceinline__ void stat_conflicts(unsigned long long* st, uint32_t c) {
  if (c == 0) return;
  atomicAdd(st + kStConflicts, (unsigned long long)c);
  atomicAdd(st + kStConflicted, 1ull);
  atomicMax(st + kStMaxConflicts, (unsigned long long)c);
  int bin = 0;
  while (bin < 9 && c > (1u << bin)) ++bin;  // 1, 2, 3-4, 5-8, ... , >256
  atomicAdd(st + kStHist + bin, 1ull);
}

__device__ __forceinline__ uint32_t ld_relaxed(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Relaxed load without a compiler memory fence: used by the filter that only
// decides whether an entry is worth an attempt (a stale value there costs an
// extra attempt, never a wrong result, since MCHD is absorbing).
__device__ __forceinline__ uint32_t ld_relaxed_nf(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p));
  return v;
}

__device__ __forceinline__ void st_relaxed(uint32_t* p, uint32_t v) {
  asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Streaming 128-bit load of four neighbour ids: read-only for the kernel's
// lifetime, not kept in L1, first to leave L2.
__device__ __forceinline__ uint4 ld_stream_v4(const uint32_t* p, uint64_t policy) {
  uint4 r;
  asm volatile(
      "ld.global.nc.L1::no_allocate.L2::cache_hint.v4.u32 {%0, %1, %2, %3}, [%4], %5;"
      : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w)
      : "l"(p), "l"(policy));
  return r;
}

__device__ __forceinline__ uint32_t ld_stream(const uint32_t* p, uint64_t policy) {
  uint32_t r;
  asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.u32 %0, [%1], %2;"
               : "=r"(r)
               : "l"(p), "l"(policy));
  return r;
}

// --- bulk copies into shared memory (the TMA engine) with an mbarrier ---
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(unsigned long long* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
// bytes (a multiple of 16) from 16-byte aligned global src to 16-byte aligned shared dst
__device__ __forceinline__ void bulk_to_smem(void* dst, const void* src, uint32_t bytes,
                                             unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ uint64_t policy_evict_first() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}

// Bounded wait with exponential back-off.  Returns false when the wait has
// run past its limit or another thread has already reported an error.
struct Waiter {
  uint64_t polls = 0;
  uint32_t ns = 32;
  __device__ __forceinline__ bool wait(const SweepParams& P) {
    ++polls;
    if (polls > P.spin_limit) {
      atomicOr(P.err, kErrTimeout);
      return false;
    }
    if ((polls & 63) == 0 && ld_relaxed(P.err) != 0) return false;
    __nanosleep(ns);
    ns = ns < 1024 ? ns * 2 : 1024;
    return true;
  }
};

// State layouts.  `raw(v)` is the 32-bit word that holds v's state (the
// whole packed word for ByteState); `matched(raw, v)` reads v's state out of
// such a word.  try_reserve / try_claim start from a word the caller has
// already observed and, when they fail, leave in it the word the CAS met, so
// a failed attempt costs no extra load.
template <int kBits>
struct PackedState {
  static constexpr uint32_t kPerWord = 32u / kBits;
  static constexpr uint32_t kMask = (1u << kBits) - 1u;
  uint32_t* words;
  uint32_t* mate;
  __device__ explicit PackedState(const SweepParams& P) : words(P.state), mate(P.mate) {}
  __device__ static __forceinline__ uint32_t word(uint32_t v) { return v / kPerWord; }
  __device__ static __forceinline__ uint32_t shift(uint32_t v) { return (v % kPerWord) * kBits; }
  __device__ __forceinline__ uint32_t raw(uint32_t v) const { return ld_relaxed(words + word(v)); }
  __device__ __forceinline__ uint32_t peek(uint32_t v) const { return ld_relaxed_nf(words + word(v)); }
  __device__ static __forceinline__ bool matched(uint32_t raw, uint32_t v) {
    return ((raw >> shift(v)) & kMask) == kMchd;
  }
  // CAS of v's field from `expect` to `desired` starting at the observed word
  // `cur`; a failure caused only by a neighbouring field is retried (it is not
  // a conflict on v).  On failure `cur` holds the word whose field for v is not
  // `expect`.
  __device__ __forceinline__ bool cas(uint32_t v, uint32_t expect, uint32_t desired, uint32_t& cur,
                                      const SweepParams& P) const {
    uint32_t* w = words + word(v);
    const uint32_t sh = shift(v);
    for (uint64_t tries = 0;; ++tries) {
      if (((cur >> sh) & kMask) != expect) return false;
      const uint32_t next = (cur & ~(kMask << sh)) | (desired << sh);
      const uint32_t old = atomicCAS(w, cur, next);
      if (old == cur) {
        cur = next;
        return true;
      }
      cur = old;
      if (tries > P.spin_limit) {  // lock-free retry; bounded all the same
        atomicOr(P.err, kErrTimeout);
        return false;
      }
    }
  }
  __device__ __forceinline__ bool try_reserve(uint32_t u, uint32_t& ru, const SweepParams& P) const {
    return cas(u, kAcc, kRsvd, ru, P);
  }
  __device__ __forceinline__ bool try_claim(uint32_t v, uint32_t /*u*/, uint32_t& rv,
                                            const SweepParams& P) const {
    return cas(v, kAcc, kMchd, rv, P);
  }
  // holder only: RSVD -> MCHD, record the pair
  __device__ __forceinline__ void commit(uint32_t u, uint32_t v) const {
    mate[u] = v;
    mate[v] = u;
    atomicXor(words + word(u), (kRsvd ^ kMchd) << shift(u));
  }
  // holder only: RSVD -> ACC
  __device__ __forceinline__ void release(uint32_t u) const {
    atomicXor(words + word(u), (kRsvd ^ kAcc) << shift(u));
  }
  // statistics instances: the same two transitions, each checked on the word
  // its atomic returns (the field must have been RSVD)
  __device__ __forceinline__ void commit_checked(uint32_t u, uint32_t v, unsigned long long* st) const {
    mate[u] = v;
    mate[v] = u;
    const uint32_t old = atomicXor(words + word(u), (kRsvd ^ kMchd) << shift(u));
    atomicAdd(st + (((old >> shift(u)) & kMask) == kRsvd ? kStTrans + 2 : kStIllegal), 1ull);
  }
  __device__ __forceinline__ void release_checked(uint32_t u, unsigned long long* st) const {
    const uint32_t old = atomicXor(words + word(u), (kRsvd ^ kAcc) << shift(u));
    atomicAdd(st + (((old >> shift(u)) & kMask) == kRsvd ? kStTrans + 3 : kStIllegal), 1ull);
  }
};

// one state byte per vertex (the paper's layout) and a 2-bit field per vertex
using ByteState = PackedState<8>;
using TwoBitState = PackedState<2>;

// words of the packed state array for n vertices at kBits per vertex
__host__ __device__ __forceinline__ uint64_t packed_words(uint64_t n, int bits) {
  const uint64_t per = 32u / (uint64_t)bits;
  return (n + per - 1) / per;
}

struct WordState {
  static constexpr uint32_t kPerWord = 1;
  uint32_t* words;
  __device__ explicit WordState(const SweepParams& P) : words(P.state) {}
  __device__ __forceinline__ uint32_t raw(uint32_t v) const { return ld_relaxed(words + v); }
  __device__ __forceinline__ uint32_t peek(uint32_t v) const { return ld_relaxed_nf(words + v); }
  __device__ static __forceinline__ bool matched(uint32_t raw, uint32_t) { return raw < kWRsvd; }
  __device__ __forceinline__ bool try_reserve(uint32_t u, uint32_t& ru, const SweepParams&) const {
    ru = atomicCAS(words + u, kWAcc, kWRsvd);
    return ru == kWAcc;
  }
  __device__ __forceinline__ bool try_claim(uint32_t v, uint32_t u, uint32_t& rv,
                                            const SweepParams&) const {
    rv = atomicCAS(words + v, kWAcc, u);
    return rv == kWAcc;
  }
  __device__ __forceinline__ void commit(uint32_t u, uint32_t v) const { st_relaxed(words + u, v); }
  __device__ __forceinline__ void release(uint32_t u) const { st_relaxed(words + u, kWAcc); }
  // statistics instances: exchanges, so the word they replace can be checked
  __device__ __forceinline__ void commit_checked(uint32_t u, uint32_t v, unsigned long long* st) const {
    const uint32_t old = atomicExch(words + u, v);
    atomicAdd(st + (old == kWRsvd ? kStTrans + 2 : kStIllegal), 1ull);
  }
  __device__ __forceinline__ void release_checked(uint32_t u, unsigned long long* st) const {
    const uint32_t old = atomicExch(words + u, kWAcc);
    atomicAdd(st + (old == kWRsvd ? kStTrans + 3 : kStIllegal), 1ull);
  }
};

// Algorithm 1, lines 6-18, for one stored entry (x, y), given words rx, ry
// already observed for x and y (they stand for the first line-10 read).
// Returns true when the row vertex x is MCHD at the end (by this attempt or by
// another thread), which lets the caller leave the rest of row x.
template <class S, bool kStats = false>
__device__ __forceinline__ bool resolve_edge(const S& s, uint32_t x, uint32_t y, uint32_t rx,
                                             uint32_t ry, const SweepParams& P) {
  if (x == y) return S::matched(rx, x);      // lines 6-7: loops are skipped
  const bool x_low = x < y;                  // lines 8-9: lower id reserved first
  const uint32_t u = x_low ? x : y, v = x_low ? y : x;
  uint32_t ru = x_low ? rx : ry, rv = x_low ? ry : rx;
  Waiter wt;
  uint32_t cnf = 0;                          // conflicts on this entry (kStats only)
  bool result = false;
  for (;;) {
    // line 10
    if (S::matched(ru, u) || S::matched(rv, v)) {
      result = S::matched(x_low ? ru : rv, x);
      break;
    }
    if (kStats && cnf == 0 && wt.polls == 0) atomicAdd(P.stats + kStAttempts, 1ull);
    if (!s.try_reserve(u, ru, P)) {          // lines 11-12: wait, then re-test line 10
      if (kStats) ++cnf;
      if (S::matched(ru, u)) {
        result = x_low;
        break;
      }
      if (!wt.wait(P)) break;
      ru = s.raw(u);
      rv = s.raw(v);
      continue;
    }
    if (kStats) atomicAdd(P.stats + kStTrans + 0, 1ull);  // ACC -> RSVD
    bool won = false, gave_up = false;
    for (;;) {                               // lines 13-16, holding u
      if (s.try_claim(v, u, rv, P)) {
        if (kStats) {
          atomicAdd(P.stats + kStTrans + 1, 1ull);  // ACC -> MCHD (v)
          s.commit_checked(u, v, P.stats);          // lines 15-16, RSVD -> MCHD (u)
        } else {
          s.commit(u, v);                      // lines 15-16
        }
        won = true;
        break;
      }
      if (kStats) ++cnf;
      if (S::matched(rv, v)) break;          // v went to another edge
      if (!wt.wait(P)) {
        gave_up = true;
        break;
      }
      rv = s.raw(v);
    }
    if (won) {
      if (kStats) atomicAdd(P.stats + kStMatches, 1ull);
      result = true;
      break;
    }
    if (kStats)
      s.release_checked(u, P.stats);         // lines 17-18, RSVD -> ACC
    else
      s.release(u);                          // lines 17-18
    result = gave_up ? false : !x_low;
    break;
  }
  if (kStats) stat_conflicts(P.stats, cnf);
  return result;
}

}  // namespace skp
